"""Pins for the FP64 oracle: each test ties it to something other than itself.

* exact optimal values (brute force over permutations, the 1-D monotone coupling,
  the translation closed form) bracket the certificate, L <= p* <= U;
* the dense primal (O-)BDRS and IPOT iterations reproduce the dual log-domain
  iterates (Lemma 1, Props. 1 and 2, App. B);
* the certificate invariants of Prop. 3 and App. F hold;
* values printed in the paper (App. F underflow example, Table 2 schedule).
Planted mistakes (in local copies of oracle functions, on the CPU) show that the
pins catch a dropped term, a wrong sign and a transposed operand.
"""
import json
import math
import os

import numpy as np
import pytest
from scipy.special import logsumexp

import oracle as O
import ot_inputs as I

GOLDEN = json.load(open(os.path.join(os.path.dirname(__file__), "golden", "paper_values.json")))


def _rand_instance(n, m, d, seed, uniform=False):
    rng = np.random.default_rng(seed)
    x = rng.random((n, d))
    y = rng.random((m, d))
    if uniform:
        r = np.full(n, 1.0 / n)
        c = np.full(m, 1.0 / m)
    else:
        r = rng.random(n) + 0.05
        c = rng.random(m) + 0.05
        r /= r.sum()
        c /= c.sum()
    return x, y, r, c


# ----------------------------------------------------------------------------------------------
# LSE and schedule
# ----------------------------------------------------------------------------------------------

def test_lse_matches_library():
    rng = np.random.default_rng(1)
    M = rng.normal(scale=300.0, size=(17, 23))
    M[3, :] -= 5000.0  # a row that underflows without the max shift
    np.testing.assert_allclose(O.lse(M, 1), logsumexp(M, axis=1), rtol=1e-14, atol=1e-12)
    np.testing.assert_allclose(O.lse(M, 0), logsumexp(M, axis=0), rtol=1e-14, atol=1e-12)


def test_schedule_matches_table2():
    g = GOLDEN["terminal_temperatures"]
    for lam, printed, num, den in zip(g["lambdas"], g["eps_T_printed"], g["eta_B_num"], g["eta_B_den"]):
        eps = O.eps_schedule(1.0, lam, g["T"])
        assert abs(eps - printed) <= 0.006e-6, (lam, eps, printed)
        # Regime 2: BDRS with eta_B = (T+1)/(lam T + 1) reaches the same terminal temperature.
        eta_b = num / den
        assert O.eps_schedule(eta_b, 1.0, g["T"]) == pytest.approx(eps, rel=1e-15)
    mi = GOLDEN["matched_iterations"]
    assert math.floor(mi["k"] / mi["lambda"]) == mi["k_O"]
    pm = GOLDEN["pixel_mass"]
    assert abs(1.0 / pm["n"] - pm["mass_printed"]) < 0.005e-7


# ----------------------------------------------------------------------------------------------
# Primal <-> dual equivalences (Lemma 1, Prop. 1, Prop. 2, App. B)
# ----------------------------------------------------------------------------------------------

@pytest.mark.parametrize("lam", [1.0, 1.2, 1.5, 1.99])
def test_primal_obdrs_equals_dual(lam):
    x, y, r, c = _rand_instance(9, 6, 2, seed=int(lam * 100))
    C = O.cost_matrix(x, y, 0.5)
    eta, iters = 1.0, 15
    P = O.primal_obdrs(r, c, C, eta, lam, iters)
    st = O.DualState.initial(9, 6)
    la, lb = np.zeros(9), np.zeros(6)
    v_prev = np.ones(6)
    for k in range(iters):
        prev = st
        st = O.dual_obdrs_step(st, np.log(r), np.log(c), C, eta, lam)
        u, v = P["u"][k], P["v"][k]
        la += lam * np.log(u)
        lb += lam * np.log(v)
        # cumulative scalings alpha^k, beta^k (Prop. 2 definitions)
        np.testing.assert_allclose(st.log_alpha, la, rtol=0, atol=1e-11)
        np.testing.assert_allclose(st.log_beta, lb, rtol=0, atol=1e-11)
        # alpha-hat^k = alpha^{k-1} u^k, beta-tilde^{k-1} = beta^{k-1} v^{k-1}, beta-hat^k = beta^{k-1} v^k
        np.testing.assert_allclose(st.log_alpha_hat, prev.log_alpha + np.log(u), atol=1e-11)
        np.testing.assert_allclose(st.log_beta_tilde, prev.log_beta + np.log(v_prev), atol=1e-11)
        np.testing.assert_allclose(st.log_beta_hat, prev.log_beta + np.log(v), atol=1e-11)
        # state X^{k+1} = diag(alpha^k) K^(lam (k+1)) diag(beta^k)
        Xd = np.exp(st.log_alpha[:, None] + st.log_beta[None, :] - lam * (k + 1) * C / eta)
        np.testing.assert_allclose(Xd, P["X"][k], rtol=1e-10, atol=0)
        v_prev = v


def test_ipot_single_inner_step_is_bdrs():
    x, y, r, c = _rand_instance(8, 11, 3, seed=7)
    C = O.cost_matrix(x, y, 1.0 / 3.0)
    eta, iters = 0.7, 20
    ip = O.ipot(r, c, C, eta, iters, inner=1)
    st = O.DualState.initial(8, 11)
    for k in range(iters):
        st = O.dual_obdrs_step(st, np.log(r), np.log(c), C, eta, 1.0)
        # Lemma 1: X^{k+1} = diag(a^k) K^(k+1) diag(b^k)
        Xd = np.exp(st.log_alpha[:, None] + st.log_beta[None, :] - (k + 1) * C / eta)
        np.testing.assert_allclose(Xd, ip["Gamma"][k], rtol=1e-10)
    # more inner steps is a different method (sanity: the pin is not vacuous)
    ip3 = O.ipot(r, c, C, eta, iters, inner=3)
    assert np.abs(ip3["Gamma"][-1] - ip["Gamma"][-1]).max() > 1e-6


def test_dual_bdrs_prop1_nonlog_form():
    """Prop. 1 written in the non-log form with (b^{k-1})^2 / b^{k-2}."""
    x, y, r, c = _rand_instance(6, 7, 2, seed=3)
    C = O.cost_matrix(x, y, 0.5)
    eta = 1.0
    a_cum, b1, b2 = np.ones(6), np.ones(7), np.ones(7)
    st = O.DualState.initial(6, 7)
    for k in range(12):
        Kk = np.exp(-(k + 1) * C / eta)
        a_cum = r / (Kk @ (b1 ** 2 / b2))
        b_new = c / (Kk.T @ a_cum)
        b2, b1 = b1, b_new
        st = O.dual_obdrs_step(st, np.log(r), np.log(c), C, eta, 1.0)
        np.testing.assert_allclose(st.log_alpha, np.log(a_cum), atol=1e-11)
        np.testing.assert_allclose(st.log_beta, np.log(b1), atol=1e-11)
        np.testing.assert_array_equal(st.log_alpha, st.log_alpha_hat)  # lam = 1: alpha = alpha-hat


# ----------------------------------------------------------------------------------------------
# Exact p* bracketing: L <= p* <= <C, Z-hat> <= U
# ----------------------------------------------------------------------------------------------

@pytest.mark.parametrize("n", [2, 3, 5, 7])
@pytest.mark.parametrize("lam", [1.0, 1.5])
def test_bruteforce_pstar_bracketed(n, lam):
    for seed in range(4):
        x, y, r, c = _rand_instance(n, n, 2, seed=100 * n + seed, uniform=True)
        C = O.cost_matrix(x, y, 0.5)
        pstar = O.pstar_bruteforce(C)
        st = O.DualState.initial(n, n)
        for k in range(60):
            st = O.dual_obdrs_step(st, np.log(r), np.log(c), C, 1.0, lam)
            if k in (0, 1, 4, 19, 59):
                cert = O.certificate_of(st, r, c, C, 1.0)
                assert cert["L"] <= pstar + 1e-12, (k, cert["L"], pstar)
                assert pstar <= cert["U"] + 1e-12, (k, cert["U"], pstar)
                Z = O.intermediate_plan(st.log_alpha_hat, st.log_beta_tilde, C, st.eps)
                Zh = O.repair(Z, r, c)
                assert Zh.min() >= -1e-15
                np.testing.assert_allclose(Zh.sum(1), r, atol=1e-13)
                np.testing.assert_allclose(Zh.sum(0), c, atol=1e-13)
                cz = float((C * Zh).sum())
                assert pstar - 1e-12 <= cz <= cert["U"] + 1e-12


def test_pstar_1d_matches_bruteforce():
    rng = np.random.default_rng(5)
    for n in range(2, 8):
        x = rng.random(n)
        y = rng.random(n)
        C = O.cost_matrix(x[:, None], y[:, None], 1.0)
        u = np.full(n, 1.0 / n)
        assert O.pstar_1d(x, u, y, u, 1.0) == pytest.approx(O.pstar_bruteforce(C), abs=1e-14)


def test_1d_nonuniform_bracketed_and_converging():
    rng = np.random.default_rng(11)
    n, m = 40, 30
    x, y = rng.random(n), rng.random(m) * 0.8 + 0.3
    r = rng.random(n) + 0.1
    c = rng.random(m) + 0.1
    r /= r.sum()
    c /= c.sum()
    kappa = 1.0 / 1.21
    C = O.cost_matrix(x[:, None], y[:, None], kappa)
    pstar = O.pstar_1d(x, r, y, c, kappa)
    res = O.solve(r, c, C, 1.0, 1.0, 3000, 100, 1.0)
    gaps = []
    for k, U, L in res["history"]:
        assert L <= pstar + 1e-12 and pstar <= U + 1e-12
        gaps.append(U - L)
    assert gaps[-1] < 0.05 * gaps[0]
    assert res["U_best"] - res["L_best"] < 0.2 * pstar


def test_translation_pstar_bracketed():
    s = 6
    z = I.grid_points(s).astype(np.float64)
    v = np.array([3.0, 1.0])
    a = I.uniform_weights(s * s, 4)
    kappa = 1.0 / (2 * (s + 3) ** 2)
    C = O.cost_matrix(z, z + v, kappa)
    pstar = O.pstar_translation(v, kappa)
    st = O.DualState.initial(s * s, s * s)
    for k in range(300):
        st = O.dual_obdrs_step(st, np.log(a), np.log(a), C, 1.0, 1.0)
        if (k + 1) % 50 == 0:
            cert = O.certificate_of(st, a, a, C, 1.0)
            assert cert["L"] <= pstar + 1e-12 <= cert["U"] + 2e-12


def test_identical_measures_pstar_zero():
    x, _, r, _ = _rand_instance(10, 10, 2, seed=9)
    C = O.cost_matrix(x, x, 0.5)
    res = O.solve(r, r, C, 1.0, 1.0, 400, 50, 1.0)
    assert res["L_best"] <= 1e-12
    assert res["U_best"] >= -1e-12


# ----------------------------------------------------------------------------------------------
# Certificate invariants (Prop. 3 proof, App. F)
# ----------------------------------------------------------------------------------------------

@pytest.mark.parametrize("lam", [1.0, 1.99])
def test_certificate_invariants(lam):
    x, y, r, c = _rand_instance(13, 9, 3, seed=21)
    C = O.cost_matrix(x, y, 1.0 / 3.0)
    st = O.DualState.initial(13, 9)
    for k in range(40):
        st = O.dual_obdrs_step(st, np.log(r), np.log(c), C, 0.5, lam)
        cert = O.certificate_of(st, r, c, C, 1.0)
        assert cert["s"].sum() == pytest.approx(1.0, abs=1e-13)
        assert np.all(cert["D"] >= 1.0) and np.all(cert["D"] <= 13.0 + 1e-12)
        assert np.all(cert["mu"] >= C.min(axis=0) - 1e-15)
        assert np.all(cert["mu"] <= C.max(axis=0) + 1e-15)
        feas = cert["f"][:, None] + cert["g"][None, :] - C
        assert feas.max() <= 1e-12
        Z = O.intermediate_plan(st.log_alpha_hat, st.log_beta_tilde, C, st.eps)
        np.testing.assert_allclose(Z.sum(1), r, rtol=1e-12)
        np.testing.assert_allclose(Z.sum(0), cert["s"], rtol=1e-11)
        assert float((C * Z).sum()) == pytest.approx(cert["cost_Z"], rel=1e-12)
        # B = c / (K^T A): log B equals log c - d
        np.testing.assert_allclose(st.log_beta_hat, np.log(c) - cert["d"], atol=1e-10)


def test_underflow_worked_example():
    g = GOLDEN["underflow_example"]
    log_A = np.array(g["log_A"])
    C = np.array(g["C_column"])[:, None]
    eps = g["eps"]
    naive = np.exp(log_A[:, None] - C / eps)
    assert np.all(naive == 0.0)  # the 0/0 the paper warns about
    cert = O.certificate(log_A, np.zeros(1), np.zeros(1), np.full(2, 0.5), np.ones(1), C, eps, 1.0)
    assert cert["mu"][0] == g["mu"]
    assert cert["M"][0] == pytest.approx(g["M"], abs=1e-12)
    assert cert["D"][0] == g["D"]
    assert cert["d"][0] == pytest.approx(g["d"], abs=1e-12)


# ----------------------------------------------------------------------------------------------
# Helpers used by large-scale spot checks and the colour cost normalisation
# ----------------------------------------------------------------------------------------------

def test_row_lse_sampled_matches_dense():
    x, y, r, c = _rand_instance(20, 300, 3, seed=2)
    C = O.cost_matrix(x, y, 0.4)
    logc = np.log(c) * 3.0
    dense = O.lse(logc[None, :] - C / 0.01, axis=1)
    rows = [0, 7, 19]
    got = O.row_lse_sampled(rows, x, y, logc, 0.4, 0.01, chunk=64)
    np.testing.assert_allclose(got, dense[rows], rtol=1e-13)


def test_max_pair_cost_hull_matches_bruteforce():
    p = I.rgb_problem(400, seed=3, m=300)
    brute = float(O.cost_matrix(p.x, p.y, 1.0).max())
    assert O.max_pair_cost_hull(p.x, p.y) == brute


# ----------------------------------------------------------------------------------------------
# Planted mistakes (in local copies, on the CPU): the pins above must catch each of them
# ----------------------------------------------------------------------------------------------

def _step_variant(st, log_r, log_c, C, eta, lam, *, momentum=True, col_uses_relaxed=False,
                  sign=1.0, transpose_col=False):
    k = st.k
    eps = O.eps_schedule(eta, lam, k)
    log_bt = st.log_beta + (sign * (st.log_beta - st.log_beta_prev) / lam if momentum else 0.0)
    log_ah = log_r - O.lse(log_bt[None, :] - C / eps, axis=1)
    log_a = (1.0 - lam) * st.log_alpha + lam * log_ah
    use = log_a if col_uses_relaxed else log_ah
    if transpose_col:
        Ct = C.T[: C.shape[0], : C.shape[1]] if C.shape[0] == C.shape[1] else C
        log_bh = log_c - O.lse(use[:, None] - Ct / eps, axis=0)
    else:
        log_bh = log_c - O.lse(use[:, None] - C / eps, axis=0)
    log_b = (1.0 - lam) * st.log_beta + lam * log_bh
    return O.DualState(log_a, log_b, st.log_beta, log_ah, log_bh, log_bt, k + 1, eps)


@pytest.mark.parametrize("mistake", [dict(momentum=False), dict(sign=-1.0),
                                     dict(col_uses_relaxed=True), dict(transpose_col=True)])
def test_planted_mistakes_break_primal_dual_pin(mistake):
    x, y, r, c = _rand_instance(7, 7, 2, seed=31)
    C = O.cost_matrix(x, y, 0.5)
    lam = 1.5
    P = O.primal_obdrs(r, c, C, 1.0, lam, 6)
    st = O.DualState.initial(7, 7)
    worst = 0.0
    for k in range(6):
        st = _step_variant(st, np.log(r), np.log(c), C, 1.0, lam, **mistake)
        Xd = np.exp(st.log_alpha[:, None] + st.log_beta[None, :] - lam * (k + 1) * C)
        worst = max(worst, np.abs(Xd - P["X"][k]).max() / P["X"][k].max())
    assert worst > 1e-6, mistake


def test_planted_mistake_dropping_repair_term_breaks_bracket():
    """Z after the first row update ignores c; its cost alone undercuts p*, the omega*delta term restores U >= p*."""
    x = np.array([0.0, 1.0])
    y = np.array([0.0, 1.0])
    r = np.array([0.5, 0.5])
    c = np.array([0.1, 0.9])
    C = O.cost_matrix(x[:, None], y[:, None], 1.0)
    pstar = O.pstar_1d(x, r, y, c, 1.0)
    assert pstar == pytest.approx(0.4)
    st = O.dual_obdrs_step(O.DualState.initial(2, 2), np.log(r), np.log(c), C, 0.1, 1.0)
    cert = O.certificate_of(st, r, c, C, 1.0)
    assert cert["cost_Z"] < pstar - 0.1          # U without omega*delta would be below p*
    assert cert["L"] <= pstar <= cert["U"]


def test_planted_mistake_wrong_eps_in_certificate_breaks_normalisation():
    """A certificate evaluated at the wrong temperature violates B = c / (K_eps^T A), the
    identity test_certificate_invariants checks."""
    x, y, r, c = _rand_instance(8, 8, 2, seed=77)
    C = O.cost_matrix(x, y, 0.5)
    st = O.dual_obdrs(r, c, C, 1.0, 1.0, 10)
    good = O.certificate_of(st, r, c, C, 1.0)
    assert np.abs(st.log_beta_hat - (np.log(c) - good["d"])).max() < 1e-10
    bad = O.certificate(st.log_alpha_hat, st.log_beta_hat, st.log_beta_tilde, r, c, C,
                        O.eps_schedule(1.0, 1.0, st.k - 2), 1.0)  # eta_{k-1} instead of eta_k
    assert np.abs(st.log_beta_hat - (np.log(c) - bad["d"])).max() > 1e-3


# ---- barycentric projection and marginal errors (App. G output; Tables 3 and 4) ----

def test_projection_closed_form_when_cost_depends_on_column_only():
    """All sources at the origin: C_ij = kappa ||y_j||^2 for every i, so each row of X is proportional
    to w_j = v_j exp(-kappa ||y_j||^2 / eps) and every source is sent to the same w-weighted mean of
    y; the row sums are u_i sum_j w_j and the column sums w_j sum_i u_i."""
    rng = np.random.default_rng(3)
    n, m, kappa, eps = 6, 9, 0.7, 0.3
    x = np.zeros((n, 2))
    y = rng.random((m, 2))
    log_u = rng.normal(size=n)
    log_v = rng.normal(size=m)
    C = O.cost_matrix(x, y, kappa)
    d = O.plan_diagnostics(log_u, log_v, C, eps, y, np.full(n, 1 / n), np.full(m, 1 / m))
    w = np.exp(log_v - kappa * (y ** 2).sum(1) / eps)
    mean = (w[:, None] * y).sum(0) / w.sum()
    assert np.allclose(d["y_hat"], mean[None, :], rtol=0, atol=1e-13)
    assert np.allclose(d["row_sums"], np.exp(log_u) * w.sum(), rtol=1e-13)
    assert np.allclose(d["col_sums"], w * np.exp(log_u).sum(), rtol=1e-13)


def test_plan_marginals_of_the_iterates():
    """From Algorithm 1's iterates: diag(A) K diag(B) with B = c / (K^T A) has column sums c, and the
    intermediate plan diag(alpha-hat) K diag(beta-tilde) has row sums r (Prop. 3; App. F); both carry
    the same total mass on either side and project inside the convex hull of the targets."""
    prob = I.grid_problem(6, 5, "gaussmix", "cauchy")
    C = O.cost_matrix(prob.x, prob.y, prob.kappa)
    a, b = prob.a, prob.b
    st = O.dual_obdrs(a, b, C, 1.0, 1.5, 40)
    Y = O.plan_diagnostics(st.log_alpha_hat, st.log_beta_hat, C, st.eps, prob.y, a, b)
    Z = O.plan_diagnostics(st.log_alpha_hat, st.log_beta_tilde, C, st.eps, prob.y, a, b)
    assert Y["col_max_rel"] < 1e-12 and Y["row_l1"] > 1e-8
    assert Z["row_max_rel"] < 1e-12
    for D in (Y, Z):
        assert abs(D["row_sums"].sum() - D["col_sums"].sum()) < 1e-13
        assert (D["y_hat"] >= prob.y.min(0) - 1e-12).all() and (D["y_hat"] <= prob.y.max(0) + 1e-12).all()
    # the sampled, on-the-fly form agrees with the dense one
    rows = np.array([0, 7, 35])
    lr, yh = O.projection_sampled(rows, prob.x, prob.y, st.log_alpha_hat, st.log_beta_hat, prob.kappa, st.eps,
                                  chunk=5)
    assert np.allclose(np.exp(lr), Y["row_sums"][rows], rtol=1e-12)
    assert np.allclose(yh, Y["y_hat"][rows], rtol=0, atol=1e-12)


# ---- annealed-Sinkhorn ablation methods (App. B; App. G "Momentum and Kernel Ablation") ----

@pytest.mark.parametrize("alg", ["bdrs", "as", "as_momentum", "as_current", "das"])
def test_ablation_log_domain_matches_multiplicative_form(alg):
    """The log-domain row/column updates reproduce the paper's multiplicative updates with Hadamard
    powers K^(k) / K^(k+1) of the base kernel (independent dense arithmetic) for every method."""
    prob = I.grid_problem(4, 8, "gaussmix", "cauchy")
    C = O.cost_matrix(prob.x, prob.y, prob.kappa)
    a, b = prob.a, prob.b
    eta, iters = 1.0, 12
    us, vs = O.ablation_primal(a, b, C, eta, iters, alg)
    st = O.DualState.initial(len(a), len(b))
    for k in range(iters):
        st = O.ablation_step(st, np.log(a), np.log(b), C, eta, alg)
        assert np.allclose(st.log_alpha_hat, np.log(us[k]), rtol=0, atol=1e-9), (alg, k)
        assert np.allclose(st.log_beta_hat, np.log(vs[k]), rtol=0, atol=1e-9), (alg, k)


def test_ablation_bdrs_corner_is_algorithm_1():
    """The current-kernel, momentum corner of the 2x2 design is Dual BDRS itself (Algorithm 1 at lam = 1)."""
    prob = I.grid_problem(5, 9, "uniform", "gaussmix")
    C = O.cost_matrix(prob.x, prob.y, prob.kappa)
    s1 = O.DualState.initial(25, 25)
    s2 = O.DualState.initial(25, 25)
    for _ in range(15):
        s1 = O.ablation_step(s1, np.log(prob.a), np.log(prob.b), C, 1.0, "bdrs")
        s2 = O.dual_obdrs_step(s2, np.log(prob.a), np.log(prob.b), C, 1.0, 1.0)
    assert np.allclose(s1.log_alpha_hat, s2.log_alpha_hat, rtol=0, atol=1e-12)
    assert np.allclose(s1.log_beta_hat, s2.log_beta_hat, rtol=0, atol=1e-12)


def test_ablation_planted_mistakes_break_the_pin():
    """A wrong kernel power or a missing debiasing factor in the log-domain step fails the primal pin."""
    prob = I.grid_problem(4, 8, "gaussmix", "cauchy")
    C = O.cost_matrix(prob.x, prob.y, prob.kappa)
    us, _ = O.ablation_primal(prob.a, prob.b, C, 1.0, 6, "das")
    us_as, _ = O.ablation_primal(prob.a, prob.b, C, 1.0, 6, "as")
    us_cur, _ = O.ablation_primal(prob.a, prob.b, C, 1.0, 6, "as_current")
    assert np.abs(np.log(us[5]) - np.log(us_as[5])).max() > 1e-3      # debiasing matters
    assert np.abs(np.log(us_as[5]) - np.log(us_cur[5])).max() > 1e-3  # kernel timing matters
    assert O.das_theta(0) == O.das_theta(1) == 0.0 and O.das_theta(4) == 0.25


# ---- rounding onto the transport polytope (the f of the paper's ablation) ----

def test_round_plan_is_feasible_and_bounds_pstar():
    """The rounded plan has exactly the prescribed marginals, is nonnegative, and its cost is at least
    p* (brute force over permutations for uniform weights); a plan already in Pi(r, c) is unchanged."""
    rng = np.random.default_rng(2)
    n = 6
    x = rng.random((n, 2)); y = rng.random((n, 2))
    C = O.cost_matrix(x, y, 1.0)
    r = c = np.full(n, 1.0 / n)
    pstar = O.pstar_bruteforce(C)
    for eps in (1.0, 0.1, 0.02):
        R = O.round_plan(rng.normal(size=n), rng.normal(size=n), C, eps, r, c)
        Z = R["Z"]
        assert (Z >= -1e-15).all()
        assert np.allclose(Z.sum(1), r, atol=1e-14) and np.allclose(Z.sum(0), c, atol=1e-14)
        assert R["cost"] >= pstar - 1e-12
    P0 = np.outer(r, c)
    R0 = O.round_plan(np.log(r), np.log(c), np.zeros((n, n)), 1.0, r, c)   # X = r c^T already feasible
    assert np.allclose(R0["Z"], P0, atol=1e-15)


def test_rank_one_correction_cost_is_separable():
    """For C_ij = kappa ||x_i - y_j||^2 the correction's cost e_r^T C e_c expands into O(n + m) sums:
    kappa [(sum e_r ||x||^2)(sum e_c) + (sum e_r)(sum e_c ||y||^2) - 2 <sum e_r x, sum e_c y>].
    (The GPU rounding relies on this; here it is checked against the dense product.)"""
    rng = np.random.default_rng(5)
    x = rng.random((7, 3)); y = rng.random((5, 3)); kappa = 0.4
    C = O.cost_matrix(x, y, kappa)
    er = rng.normal(size=7); ec = rng.normal(size=5)
    sep = kappa * ((er @ (x ** 2).sum(1)) * ec.sum() + er.sum() * (ec @ (y ** 2).sum(1)) - 2 * (er @ x) @ (ec @ y))
    assert abs(er @ C @ ec - sep) <= 1e-12


# ---- exact p* for non-uniform instances (transport LP, scipy HiGHS) ----

def test_lp_pstar_agrees_with_the_one_dimensional_closed_form():
    """Two independent exact routes agree: the LP and the monotone coupling on a line."""
    from exact_lp import lp_pstar
    rng = np.random.default_rng(8)
    x, y = rng.random(40), rng.random(30)
    a, b = rng.random(40) + 0.1, rng.random(30) + 0.1
    a, b = a / a.sum(), b / b.sum()
    C = O.cost_matrix(x[:, None], y[:, None], 1.0)
    assert abs(lp_pstar(a, b, C) - O.pstar_1d(x, a, y, b, 1.0)) <= 1e-9


@pytest.mark.parametrize("cls", ["uniform", "gaussmix", "cauchy", "sparse"])
def test_oracle_certificate_brackets_lp_pstar(cls):
    """On non-uniform grid histograms (the sparse class floored at 1e-15) the oracle's best bounds
    bracket the exact transport LP value, for BDRS and O-BDRS."""
    from exact_lp import lp_pstar
    prob = I.grid_problem(8, 21, cls, "gaussmix")
    a = np.maximum(prob.a, 1e-15); a = a / a.sum()
    b = np.maximum(prob.b, 1e-15); b = b / b.sum()
    C = O.cost_matrix(prob.x, prob.y, prob.kappa)
    pstar = lp_pstar(a, b, C)
    for lam in (1.0, 1.99):
        r = O.solve(a, b, C, 1.0, lam, 300, 50, prob.omega)
        assert r["L_best"] <= pstar + 1e-12 <= r["U_best"] + 2e-12, (cls, lam, r["L_best"], pstar, r["U_best"])


# ---- gauge (alpha c, beta / c): equivariance of Algorithm 1 and the conserved gauge step ----

def _gauge_case():
    prob = I.grid_problem(8, 41, "gaussmix", "cauchy")
    C = O.cost_matrix(prob.x, prob.y, prob.kappa)
    st = O.dual_obdrs(prob.a, prob.b, C, 1.0, 1.5, 12)
    return prob, C, st


def _shifted(st, c_alpha, c_beta, c_beta_prev):
    return O.DualState(log_alpha=st.log_alpha + c_alpha, log_beta=st.log_beta + c_beta,
                       log_beta_prev=st.log_beta_prev + c_beta_prev, log_alpha_hat=st.log_alpha_hat,
                       log_beta_hat=st.log_beta_hat, log_beta_tilde=st.log_beta_tilde, k=st.k, eps=st.eps)


@pytest.mark.parametrize("lam", [1.0, 1.5, 1.99])
def test_step_is_gauge_equivariant_and_certificate_invariant(lam):
    """A gauge c on the state (log alpha - c, log beta + c, log beta_prev + c) comes out of one
    iteration unchanged: log alpha-hat - c, log beta-hat + c, log beta + c; Prop. 3's bounds, which
    depend on the plan only, do not move."""
    prob, C, st = _gauge_case()
    la, lb = np.log(prob.a), np.log(prob.b)
    c = 37.25
    s0 = O.dual_obdrs_step(st, la, lb, C, 1.0, lam)
    s1 = O.dual_obdrs_step(_shifted(st, -c, c, c), la, lb, C, 1.0, lam)
    np.testing.assert_allclose(s1.log_alpha_hat + c, s0.log_alpha_hat, rtol=0, atol=1e-9)
    np.testing.assert_allclose(s1.log_beta_hat - c, s0.log_beta_hat, rtol=0, atol=1e-9)
    np.testing.assert_allclose(s1.log_beta - c, s0.log_beta, rtol=0, atol=1e-9)
    np.testing.assert_allclose(s1.log_alpha + c, s0.log_alpha, rtol=0, atol=1e-9)
    c0 = O.certificate_of(s0, prob.a, prob.b, C, prob.omega)
    c1 = O.certificate_of(s1, prob.a, prob.b, C, prob.omega)
    assert abs(c0["U"] - c1["U"]) <= 1e-12 and abs(c0["L"] - c1["L"]) <= 1e-12


@pytest.mark.parametrize("lam", [1.0, 1.99])
def test_momentum_conserves_a_gauge_step(lam):
    """With a gauge step v between beta^{k-2} and beta^{k-1} (log beta_prev + c, log beta + c + v),
    the momentum term log b + (log b - log b_prev) / lam carries it on: beta^k moves by c + 2v
    whatever lam is (c_k = 2 c_{k-1} - c_{k-2}), which is why O-BDRS log-scalings drift linearly."""
    prob, C, st = _gauge_case()
    la, lb = np.log(prob.a), np.log(prob.b)
    c, v = 5.0, 3.0
    s0 = O.dual_obdrs_step(st, la, lb, C, 1.0, lam)
    # alpha^{k-1} only enters through the relaxation; give it the gauge the step will produce
    s1 = O.dual_obdrs_step(_shifted(st, 0.0, c + v, c), la, lb, C, 1.0, lam)
    t_shift = (c + v) + v / lam                       # the gauge of beta-tilde
    np.testing.assert_allclose(s1.log_beta_hat - s0.log_beta_hat, t_shift, rtol=0, atol=1e-9)
    np.testing.assert_allclose(s1.log_alpha_hat - s0.log_alpha_hat, -t_shift, rtol=0, atol=1e-9)
    expect_b = (1.0 - lam) * (c + v) + lam * t_shift  # = c + 2v
    assert abs(expect_b - (c + 2 * v)) <= 1e-12
    np.testing.assert_allclose(s1.log_beta - s0.log_beta, c + 2 * v, rtol=0, atol=1e-9)
