"""The allocation-free row update, against the FP64 oracle and against ot_step's row update.

``ot_row_update_noalloc`` is for callers that may not allocate device memory (a host runtime or
plugin that owns every device allocation); it keeps its working buffers in a fixed scratch array
inside the library.  It computes

    log_alpha_hat[i] = log_r[i] - LSE_j(log_bt[j] - kappa ||x_i - y_j||^2 / eps)

and each output is checked two ways:

* against the oracle's FP64 log-sum-exp (dense ``oracle.lse`` of the cost matrix, or the oracle's
  on-the-fly ``row_lse_sampled`` on sampled rows at the capacity limit), both in cost units
  (||eps * delta||_inf / ||eps * ref||_inf <= 1e-5, the FP32-sweep tolerance of the other parity
  tests) and in log units, against a bound derived from the FP32 arithmetic of the exponent: every
  partial value of z = h_q + <A_p, w_q> (base 2) is at most Z = max|h| + sum_k max|A_k| max|w_k| in
  magnitude and takes at most d + 2 roundings of 2^-24 relative, and the log-sum-exp is
  1-Lipschitz in the per-term errors, so |delta log alpha_hat| <= ln 2 ((d + 2) 2^-24 Z + 2^-18);
* against the row update ``ot_step`` computes for the same state (the existing entry point),
  on two calls in a row that share the scratch array.

The cases cover d = 1, 2, 3, ragged sizes, the capacity limit n = m = OT_NOALLOC_MAX_POINTS, and the
documented gauge shift (log_bt - c in, output - c out).
"""
import ctypes as C

import numpy as np
import pytest

import oracle as O
import ot_inputs as I

pytestmark = pytest.mark.gpu
P = pytest.importorskip("paper_2609_33814_b300")
torch = pytest.importorskip("torch")

TOL = 1e-5
MAX_POINTS = 16384
LOG2E = 1.4426950408889634


def _fn():
    f = P.lib().ot_row_update_noalloc
    f.argtypes = [C.c_int64, C.c_int64, C.c_int32, C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p, C.c_double,
                  C.c_double, C.c_void_p, C.c_uint64]
    f.restype = C.c_int
    return f


def _call(fn, prob, log_r, log_bt, eps):
    dx = torch.from_numpy(prob.x).cuda()
    dy = torch.from_numpy(prob.y).cuda()
    dlr = torch.from_numpy(log_r).cuda()
    dbt = torch.from_numpy(np.ascontiguousarray(log_bt)).cuda()
    out = torch.full((prob.n,), float("nan"), dtype=torch.float64, device="cuda")
    torch.cuda.synchronize()
    st = fn(prob.n, prob.m, prob.d, dx.data_ptr(), dy.data_ptr(), dlr.data_ptr(), dbt.data_ptr(), prob.kappa, eps,
            out.data_ptr(), 0)
    assert st == P.OT_OK, (prob.name, st)
    return out.cpu().numpy()


def _oracle(prob, log_r, log_bt, eps, rows=None):
    """log r_i - LSE_j(log_bt_j - C_ij / eps) in FP64 (all rows, or the listed ones)."""
    if rows is None:
        C_ = O.cost_matrix(prob.x, prob.y, prob.kappa)
        return log_r - O.lse(log_bt[None, :] - C_ / eps, axis=1)
    return log_r[rows] - O.row_lse_sampled(rows, prob.x, prob.y, log_bt, prob.kappa, eps)


def _log_bound(prob, log_bt, eps):
    x = prob.x.astype(np.float64)
    y = prob.y.astype(np.float64)
    h = (log_bt - prob.kappa * (y ** 2).sum(1) / eps) * LOG2E
    A = 2.0 * prob.kappa * LOG2E / eps * np.abs(x).max(0)
    Z = np.abs(h).max() + float((A * np.abs(y).max(0)).sum())
    return np.log(2.0) * ((prob.d + 2) * 2.0 ** -24 * Z + 2.0 ** -18)


def _check(got, ref, eps, bound, what):
    err_cost = np.abs(eps * (got - ref)).max() / np.abs(eps * ref).max()
    err_log = np.abs(got - ref).max()
    assert err_cost <= TOL, (what, "cost units", err_cost)
    assert err_log <= bound, (what, "log units", err_log, bound)


def _step_reference(ctx, prob, log_bt, eps):
    """The row update of ot_step (k = 0, lambda = 1: beta-tilde = beta = log_bt, temperature eps)."""
    S = ctx.state(prob.x, prob.y, prob.a, prob.b, cost_scale=prob.kappa, omega=prob.omega, eps0=eps, lam=1.0,
                  cert_every=0)
    S.set(P.OT_LOG_BETA, log_bt, 0)
    S.set(P.OT_LOG_BETA_PREV, log_bt, 0)
    S.step(1)
    out = S.get(P.OT_LOG_ALPHA_HAT)
    S.close()
    return out


def _cases():
    g = I.grid_problem(32, 7, "gaussmix", "uniform")
    x = I.random_cloud(3000, 3, 8)
    y = I.random_cloud(2000, 3, 9)
    r3 = I.Problem(x, y, I.uniform_weights(3000, 10), I.uniform_weights(2000, 11), 1.0 / 3.0, 1.0, "ragged3")
    x1 = I.random_cloud(777, 1, 12)
    y1 = I.random_cloud(1500, 1, 13)
    r1 = I.Problem(x1, y1, I.uniform_weights(777, 14), I.uniform_weights(1500, 15), 1.0, 1.0, "line")
    return [(g, 0.05), (r3, 0.02), (r1, 0.01)]


def test_noalloc_row_update_matches_oracle_and_step_twice():
    fn = _fn()
    ctx = P.Context(0)
    rng = np.random.default_rng(3)
    for prob, eps in _cases():
        log_r = np.log(prob.a / prob.a.sum())
        for call in range(2):  # two calls in a row share the scratch array
            log_bt = rng.normal(0.0, 3.0, prob.m) / eps * 0.01
            got = _call(fn, prob, log_r, log_bt, eps)
            bound = _log_bound(prob, log_bt, eps)
            _check(got, _oracle(prob, log_r, log_bt, eps), eps, bound, (prob.name, call, "oracle"))
            ref = _step_reference(ctx, prob, log_bt, eps)
            err = np.abs(eps * (got - ref)).max() / np.abs(eps * ref).max()
            assert err <= TOL, (prob.name, call, "ot_step", err)
    ctx.close()


def test_noalloc_at_capacity_sampled_rows():
    """n = m = OT_NOALLOC_MAX_POINTS (a 128 x 128 grid): every point block and the full split count of
    the fixed scratch layout are in use; sampled rows (the last ones included) against the oracle."""
    fn = _fn()
    prob = I.grid_problem(128, 31, "cauchy", "gaussmix")
    assert prob.n == MAX_POINTS and prob.m == MAX_POINTS
    eps = 2e-3
    log_r = np.log(prob.a / prob.a.sum())
    rng = np.random.default_rng(4)
    rows = np.unique(np.concatenate([rng.choice(prob.n, 40, replace=False), np.arange(prob.n - 8, prob.n)]))
    for call in range(2):
        log_bt = rng.normal(0.0, 1.0, prob.m)
        got = _call(fn, prob, log_r, log_bt, eps)
        assert np.isfinite(got).all()
        _check(got[rows], _oracle(prob, log_r, log_bt, eps, rows), eps, _log_bound(prob, log_bt, eps),
               ("capacity", call))


def test_noalloc_gauge_shift():
    """A drifted gauge (log_bt + 3e5) passed as log_bt - c with c = its first entry: the output is the
    row update of the drifted log_bt plus c (LSE_j(log_bt_j - c - C_ij/eps) = LSE_j(...) - c), so the
    output - c matches the drifted row update at the accuracy of an undrifted one."""
    fn = _fn()
    prob, eps = _cases()[0]
    log_r = np.log(prob.a / prob.a.sum())
    log_bt = np.random.default_rng(5).normal(0.0, 3.0, prob.m) / eps * 0.01 + 3.0e5
    c = float(log_bt[0])
    got = _call(fn, prob, log_r, log_bt - c, eps) - c
    ref = _oracle(prob, log_r, log_bt, eps)
    bound = _log_bound(prob, log_bt - c, eps)
    assert np.abs(got - ref).max() <= bound, (np.abs(got - ref).max(), bound)


def test_noalloc_rejects_sizes_beyond_its_scratch():
    fn = _fn()
    n = MAX_POINTS + 1
    x = torch.zeros((n, 2), dtype=torch.float32, device="cuda")
    lr = torch.zeros(n, dtype=torch.float64, device="cuda")
    out = torch.zeros(n, dtype=torch.float64, device="cuda")
    st = fn(n, 4, 2, x.data_ptr(), x.data_ptr(), lr.data_ptr(), lr.data_ptr(), 1.0, 1.0, out.data_ptr(), 0)
    assert st == P.OT_EINVAL
    st = fn(4, n, 2, x.data_ptr(), x.data_ptr(), lr.data_ptr(), lr.data_ptr(), 1.0, 1.0, out.data_ptr(), 0)
    assert st == P.OT_EINVAL
