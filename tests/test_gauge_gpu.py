"""Large gauge in the log-scalings.

The iteration of Algorithm 1 carries the gauge (alpha c, beta / c) along unchanged, and its
momentum term keeps a gauge step per iteration (log beta^k - log beta^{k-1}) constant. O-BDRS runs
therefore drift linearly: on 16x16 grid histograms at lambda = 1.99 the oracle's log beta passes
4e5 by iteration 7000 while the plan stays put.  The FP32 sweeps must stay as accurate there as at
k = 0, which is what the pack offsets are for.

* One-step parity from a state shifted by a gauge of +-3e5 (via ot_state_set): the GPU's step,
  with the gauge taken back out, against the oracle's step from the unshifted state, at the
  FP32 tolerance (1e-5 of the potential scale); the certificate bounds, which are gauge-invariant,
  at 1e-6.
* Long O-BDRS runs (lambda = 1.99, 10^4 iterations) on the 16x16 grid pairs where an FP32 pack
  without offsets lost the gauge to rounding and overflowed: every certificate stays finite and
  brackets the exact transport LP value.
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


def _gauged_gpu_state(ctx, prob, st, c, lam, precision, cert_every):
    S = ctx.state(prob.x, prob.y, prob.a, prob.b, cost_scale=prob.kappa, omega=prob.omega, eps0=1.0, lam=lam,
                  precision=precision, cert_every=cert_every, max_iters=10 ** 6)
    S.set(P.OT_LOG_ALPHA, st.log_alpha - c, st.k)
    S.set(P.OT_LOG_BETA, st.log_beta + c, st.k)
    S.set(P.OT_LOG_BETA_PREV, st.log_beta_prev + c, st.k)
    return S


@pytest.mark.parametrize("precision", ["mufu", "split", "comp"])
@pytest.mark.parametrize("c", [3e5, -3e5])
@pytest.mark.parametrize("lam,k0", [(1.99, 40), (1.0, 100)])
def test_one_step_parity_under_large_gauge(ctx, precision, c, lam, k0):
    prob = I.grid_problem(16, 31, "gaussmix", "sparse")
    a = np.maximum(prob.a, 1e-15)
    a = a / a.sum()
    b = np.maximum(prob.b, 1e-15)
    b = b / b.sum()
    C = O.cost_matrix(prob.x, prob.y, prob.kappa)
    st0 = O.dual_obdrs(a, b, C, 1.0, lam, k0)
    st1 = O.dual_obdrs_step(st0, np.log(a), np.log(b), C, 1.0, lam)
    S = _gauged_gpu_state(ctx, I.Problem(prob.x, prob.y, a, b, prob.kappa, prob.omega, "g"), st0, c, lam,
                          precision, cert_every=0)
    S.step(1)
    eps = st1.eps
    f_o, g_o = eps * st1.log_alpha_hat, eps * (st1.log_beta_hat - np.log(b))
    f_g = eps * (S.get(P.OT_LOG_ALPHA_HAT) + c)
    g_g = eps * (S.get(P.OT_LOG_BETA_HAT) - c - np.log(b))
    scale = max(np.abs(f_o).max(), np.abs(g_o).max())
    err = max(np.abs(f_g - f_o).max(), np.abs(g_g - g_o).max()) / scale
    assert err <= 1e-5, (precision, c, err)
    S.close()


@pytest.mark.parametrize("c", [3e5, -3e5])
def test_certificate_under_large_gauge(ctx, c):
    prob = I.grid_problem(16, 32, "cauchy", "gaussmix")
    C = O.cost_matrix(prob.x, prob.y, prob.kappa)
    st0 = O.dual_obdrs(prob.a, prob.b, C, 1.0, 1.99, 60)
    st1 = O.dual_obdrs_step(st0, np.log(prob.a), np.log(prob.b), C, 1.0, 1.99)
    cert_o = O.certificate_of(st1, prob.a, prob.b, C, prob.omega)
    S = _gauged_gpu_state(ctx, prob, st0, c, 1.99, "mufu", cert_every=1)
    res = S.step(1)
    assert abs(res["U"] - cert_o["U"]) <= 1e-6, (res["U"], cert_o["U"])
    assert abs(res["L"] - cert_o["L"]) <= 1e-6, (res["L"], cert_o["L"])
    S.close()


# 16x16 grid pairs (seed, source class, target class) of the certification-delay workload on which
# O-BDRS at lambda = 1.99 overflowed between iterations 6880 and 9940 before the pack offsets
DRIFT_CASES = [(2609 + 4, "cauchy", "sparse"), (2609 + 6, "sparse", "uniform"), (2609 + 10, "gaussmix", "cauchy"),
               (2609 + 12, "cauchy", "sparse"), (2609 + 14, "sparse", "uniform")]


@pytest.mark.parametrize("seed,ca,cb", DRIFT_CASES)
def test_long_obdrs_run_stays_finite_and_brackets_lp(ctx, seed, ca, cb):
    from exact_lp import lp_pstar
    prob = I.grid_problem(16, seed, ca, cb)
    a = np.maximum(prob.a, 1e-15)
    a = a / a.sum()
    b = np.maximum(prob.b, 1e-15)
    b = b / b.sum()
    pstar = lp_pstar(a, b, O.cost_matrix(prob.x, prob.y, prob.kappa))
    S = ctx.state(prob.x, prob.y, prob.a, prob.b, cost_scale=prob.kappa, omega=1.0, zero_mass_floor=1e-15,
                  eps0=1.0, lam=1.99, precision="mufu", cert_every=100)
    for _ in range(10):
        res = S.step(1000)
        assert np.isfinite(res["U"]) and np.isfinite(res["L"])
        assert res["L_best"] <= pstar + 1e-6 and pstar <= res["U_best"] + 1e-6, (res["L_best"], pstar, res["U_best"])
    # the gauge did drift (the case is the one it is meant to be), and the plan converged
    drift = np.abs(S.get(P.OT_LOG_BETA)).max()
    assert drift > 1e5, drift
    assert res["U_best"] - res["L_best"] < 1e-3, (res["U_best"], res["L_best"])
    S.close()
