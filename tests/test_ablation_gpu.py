"""The annealed-Sinkhorn ablation methods (App. B; App. G "Momentum and Kernel Ablation") on the GPU
against the oracle's log-domain steps (themselves pinned to the paper's multiplicative updates).

Tolerances as for Algorithm 1: one-step potentials at 1e-5 (FP32 sweeps) / 1e-9 (FP64), full FP64
trajectories at 1e-9, all relative to max(|f|, |g|)."""
import numpy as np
import pytest

import oracle as O
import ot_inputs as I

pytestmark = pytest.mark.gpu
P = pytest.importorskip("paper_2609_33814_b300")

ALGS = ["bdrs", "as", "as_momentum", "as_current", "das"]
TOL = {"mufu": 1e-5, "fp64": 1e-9}


@pytest.fixture(scope="module")
def ctx():
    return P.Context(0)


def _err(st, lah, lbh, logc):
    f_o, g_o = st.eps * st.log_alpha_hat, st.eps * (st.log_beta_hat - logc)
    scale = max(np.abs(f_o).max(), np.abs(g_o).max())
    return max(np.abs(st.eps * lah - f_o).max(), np.abs(st.eps * (lbh - logc) - g_o).max()) / scale


@pytest.mark.parametrize("precision", ["mufu", "fp64"])
@pytest.mark.parametrize("alg", ALGS)
@pytest.mark.parametrize("k0", [0, 1, 5])
def test_one_step(ctx, alg, precision, k0):
    prob = I.grid_problem(16, 40 + k0, "gaussmix", "cauchy")
    C = O.cost_matrix(prob.x, prob.y, prob.kappa)
    a, b = prob.a / prob.a.sum(), prob.b / prob.b.sum()
    st = O.DualState.initial(len(a), len(b))
    for _ in range(k0):
        st = O.ablation_step(st, np.log(a), np.log(b), C, 1.0, alg)
    S = ctx.state(prob.x, prob.y, prob.a, prob.b, cost_scale=prob.kappa, omega=prob.omega, eps0=1.0,
                  precision=precision, cert_every=0, algorithm=alg)
    if k0 > 0:
        S.set(P.OT_LOG_ALPHA, st.log_alpha, k0)
        S.set(P.OT_LOG_BETA, st.log_beta, k0)
        S.set(P.OT_LOG_BETA_PREV, st.log_beta_prev, k0)
    st1 = O.ablation_step(st, np.log(a), np.log(b), C, 1.0, alg)
    S.step(1)
    assert _err(st1, S.get(P.OT_LOG_ALPHA_HAT), S.get(P.OT_LOG_BETA_HAT), np.log(b)) <= TOL[precision]
    S.close()


@pytest.mark.parametrize("alg", ALGS)
def test_fp64_trajectory(ctx, alg):
    prob = I.grid_problem(16, 7, "uniform", "gaussmix")
    C = O.cost_matrix(prob.x, prob.y, prob.kappa)
    a, b = prob.a / prob.a.sum(), prob.b / prob.b.sum()
    st = O.DualState.initial(len(a), len(b))
    for _ in range(150):
        st = O.ablation_step(st, np.log(a), np.log(b), C, 1.0, alg)
    S = ctx.state(prob.x, prob.y, prob.a, prob.b, cost_scale=prob.kappa, omega=prob.omega, eps0=1.0,
                  precision="fp64", cert_every=0, algorithm=alg)
    S.step(150)
    assert _err(st, S.get(P.OT_LOG_ALPHA_HAT), S.get(P.OT_LOG_BETA_HAT), np.log(b)) <= 1e-9
    S.close()


def test_rules_and_current_kernel_certificate(ctx):
    prob = I.grid_problem(12, 3)
    kw = dict(cost_scale=prob.kappa, omega=prob.omega)
    for bad in (dict(algorithm="as", lam=1.5, cert_every=0), dict(algorithm="das", cert_every=10),
                dict(algorithm="as_momentum", cert_every=5)):
        with pytest.raises(P.OTError) as e:
            ctx.state(prob.x, prob.y, prob.a, prob.b, **kw, **bad)
        assert e.value.status == P.OT_EINVAL
    S = ctx.state(prob.x, prob.y, prob.a, prob.b, **kw, algorithm="as", cert_every=0)
    S.step(5)
    with pytest.raises(P.OTError) as e:
        S.certificate()
    assert e.value.status == P.OT_EINVAL
    S.close()
    # a current-kernel method keeps a valid certificate: L <= p* <= U on an exactly solvable instance
    x = I.random_cloud(200, 1, 1)
    y = I.random_cloud(150, 1, 2)
    a, b = I.uniform_weights(200, 3), I.uniform_weights(150, 4)
    pstar = O.pstar_1d(x[:, 0], a, y[:, 0], b, 1.0)
    f, g, res = ctx.solve(x, y, a, b, cost_scale=1.0, omega=1.0, max_iters=300, cert_every=50,
                          algorithm="as_current")
    assert res["n_certs"] == 6 and res["L_best"] <= pstar + 1e-12 <= res["U_best"] + 2e-12
