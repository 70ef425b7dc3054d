"""FP64 CPU oracle for Dual (O-)BDRS and its primal-dual certificate.

TEST INFRASTRUCTURE ONLY.  Nothing in the product path may import this module:
only the tests, the smoke check and the benchmark's CPU-baseline leg use it.
It shares no code with the CUDA path (no kernels, helpers, constants or
pre-/post-processing); the only module both sides use is ``ot_inputs``, which
draws seeded inputs and holds none of the method's arithmetic.

Everything here is plain, slow, dense FP64 numpy, written to be checked
against the paper by eye:

* ``cost_matrix``            - C_ij = kappa ||x_i - y_j||^2 (Sec. 2; App. G cost construction)
* ``lse``                    - LSE as defined beside Algorithm 1, two-pass max-shifted
* ``dual_obdrs_step``        - one iteration of Algorithm 1 (Dual O-BDRS, log domain)
* ``ablation_step``          - the annealed-Sinkhorn ablation methods (AS, AS with momentum,
                               current-kernel AS, DAS; App. B, App. G), log domain, and
  ``ablation_primal``          their multiplicative forms with Hadamard powers of K
* ``certificate``            - Proposition 3 with the stabilised upper bound of Algorithm 2
* ``repair``                 - the feasible repair Z-hat from the proof of Proposition 3
* ``primal_obdrs``           - primal (O-)BDRS, Eq. (bdrs) and Eq. (o_bdrs_x), dense non-log
* ``ipot``                   - IPOT with L inner Sinkhorn steps (App. B); L=1 is BDRS
* ``pstar_*``                - exact OT values used as pins (brute force, 1-D, translation)
* ``solve``                  - Algorithm 1 with periodic certificates and best-so-far bounds
* ``row_lse_sampled``        - on-the-fly FP64 row LSE for a sample of rows (large instances)
* ``plan_diagnostics``       - barycentric projection and marginal errors of an implicit plan
                               (App. G "Implicit implementation and output"; Tables 3 and 4)
* ``projection_sampled``     - the same projection for a sample of rows, costs on the fly
* ``round_plan``             - rounding of an implicit plan onto the transport polytope (the
                               Altschuler-Weed-Rigollet procedure the paper's ablation uses for f)

Pins (tests that tie this oracle to something other than itself) live in
``tests/test_oracle_pins.py``: brute-force p* over permutations, the 1-D
monotone coupling, the translation closed form, primal IPOT/(O-)BDRS against
the dual iteration, the certificate invariants of Proposition 3 and
Appendix F, the underflow example of Appendix F and the schedule values of
Table 2.  Every function below is covered by at least one of them.
"""
from __future__ import annotations

import dataclasses
import itertools
import math
from typing import Optional

import numpy as np


# --------------------------------------------------------------------------------------------
# Cost and LSE
# --------------------------------------------------------------------------------------------

def cost_matrix(x: np.ndarray, y: np.ndarray, kappa: float) -> np.ndarray:
    """Dense C_ij = kappa * ||x_i - y_j||^2 in FP64 (difference form, no expansion).

    Squared-Euclidean ground cost of the paper's experiments (App. G: grid cost
    ||z_i - z_j||^2 / (2(s-1)^2); colour cost ||x_i - y_j||^2 / max_pq ||x_p - y_q||^2).
    """
    x = np.asarray(x, dtype=np.float64)
    y = np.asarray(y, dtype=np.float64)
    diff = x[:, None, :] - y[None, :, :]
    return kappa * np.einsum("ijk,ijk->ij", diff, diff)


def lse(M: np.ndarray, axis: int) -> np.ndarray:
    """log sum exp along ``axis`` (Algorithm 1: [LSE(M)]_p = log sum_q exp(M_pq)).

    Two passes: the exact maximum, then the sum of exp(M - max).
    """
    mx = np.max(M, axis=axis, keepdims=True)
    mx_safe = np.where(np.isfinite(mx), mx, 0.0)
    s = np.sum(np.exp(M - mx_safe), axis=axis, keepdims=True)
    out = mx_safe + np.log(s)
    return np.squeeze(out, axis=axis)


def eps_schedule(eta: float, lam: float, k: int) -> float:
    """Effective temperature eta_k = eta / (lam*k + 1) (Algorithm 1; Prop. 2: K_k^O = K^(lam k + 1))."""
    return eta / (lam * k + 1.0)


# --------------------------------------------------------------------------------------------
# Algorithm 1: Dual O-BDRS in the log domain
# --------------------------------------------------------------------------------------------

@dataclasses.dataclass
class DualState:
    """State of Algorithm 1 after ``k`` completed iterations.

    ``log_beta`` is log beta^{k-1} and ``log_beta_prev`` is log beta^{k-2} as seen by the
    *next* iteration; the hatted and tilded vectors are those of the last completed
    iteration (its return tuple), and ``eps`` is that iteration's eta_k.
    """
    log_alpha: np.ndarray
    log_beta: np.ndarray
    log_beta_prev: np.ndarray
    log_alpha_hat: np.ndarray
    log_beta_hat: np.ndarray
    log_beta_tilde: np.ndarray
    k: int = 0
    eps: float = float("nan")

    @staticmethod
    def initial(n: int, m: int) -> "DualState":
        """Algorithm 1 initialisation: log alpha^{-1} = log beta^{-2} = log beta^{-1} = 0."""
        z = np.zeros
        return DualState(z(n), z(m), z(m), z(n), z(m), z(m), 0, float("nan"))

    def copy(self) -> "DualState":
        return DualState(*(np.array(v, copy=True) if isinstance(v, np.ndarray) else v
                           for v in dataclasses.astuple(self)))


def dual_obdrs_step(st: DualState, log_r: np.ndarray, log_c: np.ndarray, C: np.ndarray,
                    eta: float, lam: float) -> DualState:
    """One iteration k of Algorithm 1 (Dual O-BDRS, log domain); lam = 1 is Dual BDRS.

    eta_k   = eta/(lam k + 1)
    log bt  = log b^{k-1} + (1/lam)(log b^{k-1} - log b^{k-2})          (momentum)
    log ah  = log r - LSE_j(log bt_j - C_ij/eta_k)                        (row update)
    log a   = (1-lam) log a^{k-1} + lam log ah                             (relaxation)
    log bh  = log c - LSE_i(log ah_i - C_ij/eta_k)                        (column update, uses ah)
    log b   = (1-lam) log b^{k-1} + lam log bh                             (relaxation)
    """
    k = st.k
    eps = eps_schedule(eta, lam, k)
    log_bt = st.log_beta + (st.log_beta - st.log_beta_prev) / lam
    log_ah = log_r - lse(log_bt[None, :] - C / eps, axis=1)
    log_a = (1.0 - lam) * st.log_alpha + lam * log_ah
    log_bh = log_c - lse(log_ah[:, None] - C / eps, axis=0)
    log_b = (1.0 - lam) * st.log_beta + lam * log_bh
    return DualState(log_alpha=log_a, log_beta=log_b, log_beta_prev=st.log_beta,
                     log_alpha_hat=log_ah, log_beta_hat=log_bh, log_beta_tilde=log_bt,
                     k=k + 1, eps=eps)


# Annealed-Sinkhorn ablation (App. B "Annealed Sinkhorn Detailed Comparison", App. G "Momentum and
# Kernel Ablation"): methods that differ from Dual BDRS only in the row update, under the same
# inverse-linear schedule (lam = 1):
#   kernel   "old": K^(k) = exp(-C / eta_{k-1}) (eta_{-1} = infinity: K^(0) = 1), "current": K^(k+1)
#   scaling  no momentum: v^{k-1};  momentum: (v^{k-1})^2 / v^{k-2}
#   DAS      old kernel, no momentum, numerator (u^{k-1})^theta_k r with theta_1 = 0, theta_k = 1/k
ALGORITHMS = {
    "bdrs": ("current", True, False),
    "as": ("old", False, False),
    "as_momentum": ("old", True, False),
    "as_current": ("current", False, False),
    "das": ("old", False, True),
}


def das_theta(k: int) -> float:
    """theta_k = 1 - eta_{k-1} / eta_{max(k-2, 0)} under eta_k = eta / (k + 1): 0 for k <= 1, 1/k after."""
    return 0.0 if k <= 1 else 1.0 / k


def ablation_step(st: DualState, log_r, log_c, C, eta: float, algorithm: str) -> DualState:
    """One iteration k of an ablation method in the log domain (lam = 1, so alpha = alpha-hat)."""
    kernel, momentum, debias = ALGORITHMS[algorithm]
    k = st.k
    eps = eps_schedule(eta, 1.0, k)                                  # column update: current kernel
    inv_row = (k / eta) if kernel == "old" else (1.0 / eps)          # 1 / eta_{k-1} (0 at k = 0) or 1 / eta_k
    log_bt = st.log_beta + (st.log_beta - st.log_beta_prev) if momentum else st.log_beta.copy()
    log_ah = log_r - lse(log_bt[None, :] - C * inv_row, axis=1)
    if debias:
        log_ah = log_ah + das_theta(k) * st.log_alpha
    log_bh = log_c - lse(log_ah[:, None] - C / eps, axis=0)
    return DualState(log_alpha=log_ah, log_beta=log_bh, log_beta_prev=st.log_beta, log_alpha_hat=log_ah,
                     log_beta_hat=log_bh, log_beta_tilde=log_bt, k=k + 1, eps=eps)


def ablation_primal(r, c, C, eta: float, iters: int, algorithm: str):
    """The same methods in the paper's multiplicative form with dense Hadamard powers of K = exp(-C/eta)
    (small problems only): returns the lists of scalings u^k, v^k."""
    kernel, momentum, debias = ALGORITHMS[algorithm]
    K = np.exp(-np.asarray(C, np.float64) / eta)
    u_prev = np.ones(len(r))
    v1 = np.ones(len(c))   # v^{k-1}
    v2 = np.ones(len(c))   # v^{k-2}
    us, vs = [], []
    for k in range(iters):
        Krow = K ** k if kernel == "old" else K ** (k + 1)
        vin = v1 * v1 / v2 if momentum else v1
        num = r * (u_prev ** das_theta(k) if debias else 1.0)
        u = num / (Krow @ vin)
        v = c / ((K ** (k + 1)).T @ u)
        us.append(u)
        vs.append(v)
        u_prev, v2, v1 = u, v1, v
    return us, vs


def dual_obdrs(r, c, C, eta, lam, iters, state: Optional[DualState] = None) -> DualState:
    """``iters`` iterations of Algorithm 1 from ``state`` (default: the initialisation)."""
    st = DualState.initial(len(r), len(c)) if state is None else state
    log_r, log_c = np.log(r), np.log(c)
    for _ in range(iters):
        st = dual_obdrs_step(st, log_r, log_c, C, eta, lam)
    return st


# --------------------------------------------------------------------------------------------
# Proposition 3 + Algorithm 2: the certificate
# --------------------------------------------------------------------------------------------

def certificate(log_A, log_B, log_t, r, c, C, eps, omega) -> dict:
    """Primal-dual certificate of Proposition 3, upper bound evaluated as in Algorithm 2.

    Inputs are the shared scalings of the certificate table (Sec. 3.4): for O-BDRS
    A = alpha-hat^k, B = beta-hat^k, t = beta-tilde^{k-1}, eps = eta/(lam k + 1).

    Lower bound:  f = eps log A,  g = eps log(B/c),  L = <r,f> + <c,g>.
    Upper bound (Algorithm 2), per column j:
        l_i = log A_i - C_ij/eps,  M_j = max_i l_i,  E_i = exp(l_i - M_j),
        D_j = sum E,  N_j = sum C_ij E_i,  mu_j = N_j/D_j,  d_j = M_j + log D_j,
        s_j = exp(log t_j + d_j);
    then delta = 1/2 sum_j |s_j - c_j| and U = sum_j s_j mu_j + omega delta.
    """
    log_A = np.asarray(log_A, np.float64)
    log_B = np.asarray(log_B, np.float64)
    log_t = np.asarray(log_t, np.float64)
    f = eps * log_A
    g = eps * (log_B - np.log(c))
    L = float(np.dot(r, f) + np.dot(c, g))
    ell = log_A[:, None] - C / eps
    M = ell.max(axis=0)
    E = np.exp(ell - M[None, :])
    D = E.sum(axis=0)
    N = (C * E).sum(axis=0)
    mu = N / D
    d = M + np.log(D)
    s = np.exp(log_t + d)
    delta = 0.5 * float(np.abs(s - c).sum())
    cost_Z = float(np.dot(s, mu))
    U = cost_Z + omega * delta
    return dict(U=U, L=L, gap=U - L, delta=delta, cost_Z=cost_Z, f=f, g=g, s=s, mu=mu,
                D=D, N=N, M=M, d=d)


def certificate_of(st: DualState, r, c, C, omega) -> dict:
    """Certificate of the last completed iteration of ``st`` (O-BDRS row of the table)."""
    return certificate(st.log_alpha_hat, st.log_beta_hat, st.log_beta_tilde, r, c, C, st.eps, omega)


def intermediate_plan(log_A, log_t, C, eps) -> np.ndarray:
    """Z = diag(A) K_eps diag(t), the plan right after the row update (Sec. 3.4)."""
    return np.exp(np.asarray(log_A)[:, None] - C / eps + np.asarray(log_t)[None, :])


def repair(Z: np.ndarray, r: np.ndarray, c: np.ndarray) -> np.ndarray:
    """Feasible repair Z-hat of a row-feasible plan Z (proof of Proposition 3).

    Clip over-full columns by e_j = min(1, c_j/s_j), then add p q^T / delta with the
    remaining row and column deficits p, q.
    """
    s = Z.sum(axis=0)
    delta = 0.5 * float(np.abs(s - c).sum())
    if delta == 0.0:
        return Z.copy()
    e = np.minimum(1.0, c / s)
    Zt = Z * e[None, :]
    p = r - Zt.sum(axis=1)
    q = c - Zt.sum(axis=0)
    return Zt + np.outer(p, q) / delta


# --------------------------------------------------------------------------------------------
# Primal forms (dense, non-log): BDRS, O-BDRS and IPOT
# --------------------------------------------------------------------------------------------

def primal_obdrs(r, c, C, eta, lam, iters) -> dict:
    """Primal-dual (O-)BDRS with a dense plan, Eq. (bdrs) and Eq. (o_bdrs_x).

    K = exp(-C/eta), X^0 = 1, v^{-1} = 1;
      u^k = r / ((X^k . K) v^{k-1}),   v^k = c / ((X^k . K)^T u^k),
      X^{k+1} = X^k . (K . u^k (v^k)^T)^lam      (lam = 1: diag(u)(X.K)diag(v)).
    Returns the per-iteration u, v and the plans X^{k+1}.
    """
    K = np.exp(-C / eta)
    X = np.ones_like(C)
    v = np.ones(C.shape[1])
    us, vs, Xs = [], [], []
    for _ in range(iters):
        Q = X * K
        u = r / (Q @ v)
        v = c / (Q.T @ u)
        X = X * (K * np.outer(u, v)) ** lam
        us.append(u)
        vs.append(v)
        Xs.append(X.copy())
    return dict(u=us, v=vs, X=Xs)


def ipot(mu, nu, C, eta, outer, inner=1) -> dict:
    """IPOT (App. B, after Xie et al.): proximal point with ``inner`` Sinkhorn steps.

    G = exp(-C/eta), Gamma^(1) = 1, b = 1; each outer step t:
      Q = Gamma^(t) . G;  repeat ``inner`` times: a = mu/(Q b), b = nu/(Q^T a);
      Gamma^(t+1) = diag(a) Q diag(b).
    With inner = 1 this is warm-started single-inner-iteration IPOT.
    """
    G = np.exp(-C / eta)
    Gam = np.ones_like(C)
    b = np.ones(C.shape[1])
    As, Bs, Gs = [], [], []
    for _ in range(outer):
        Q = Gam * G
        for _ in range(inner):
            a = mu / (Q @ b)
            b = nu / (Q.T @ a)
        Gam = a[:, None] * Q * b[None, :]
        As.append(a)
        Bs.append(b)
        Gs.append(Gam.copy())
    return dict(a=As, b=Bs, Gamma=Gs)


# --------------------------------------------------------------------------------------------
# Exact p* for pins
# --------------------------------------------------------------------------------------------

def pstar_bruteforce(C: np.ndarray) -> float:
    """p* for uniform weights and n = m <= 8: the best permutation, (1/n) min_sigma sum C_{i sigma(i)}.

    Birkhoff-von Neumann: with uniform marginals the transportation polytope's
    vertices are permutation matrices scaled by 1/n.
    """
    n = C.shape[0]
    assert C.shape == (n, n) and n <= 8
    best = math.inf
    idx = np.arange(n)
    for perm in itertools.permutations(range(n)):
        v = float(C[idx, list(perm)].sum())
        best = min(best, v)
    return best / n


def pstar_1d(x, a, y, b, kappa) -> float:
    """p* on the real line for convex cost kappa |x - y|^2: the monotone (quantile) coupling.

    Sort both supports and walk the two cumulative distributions (north-west
    corner rule on the sorted supports), moving the smaller remaining mass each step.
    """
    ox, oy = np.argsort(x, kind="stable"), np.argsort(y, kind="stable")
    xs, ws = np.asarray(x, np.float64)[ox], np.asarray(a, np.float64)[ox].copy()
    ys, vs = np.asarray(y, np.float64)[oy], np.asarray(b, np.float64)[oy].copy()
    i = j = 0
    total = 0.0
    while i < len(xs) and j < len(ys):
        mass = min(ws[i], vs[j])
        total += mass * kappa * (xs[i] - ys[j]) ** 2
        ws[i] -= mass
        vs[j] -= mass
        if ws[i] <= vs[j]:
            i += 1
        else:
            j += 1
    return total


def pstar_translation(v, kappa) -> float:
    """p* between a measure and its translate by v under kappa ||.||^2: kappa ||v||^2."""
    v = np.asarray(v, np.float64)
    return float(kappa * np.dot(v, v))


def max_pair_cost_hull(x: np.ndarray, y: np.ndarray) -> float:
    """Exact max_{p,q} ||x_p - y_q||^2 in FP64 (App. G colour-cost normalisation).

    ||x - y||^2 is convex in each argument, so the maximum over two point sets is
    attained at vertices of their convex hulls; brute force over hull vertices.
    """
    from scipy.spatial import ConvexHull

    def verts(p):
        p = np.asarray(p, np.float64)
        try:
            return p[ConvexHull(p).vertices]
        except Exception:
            return p
    hx, hy = verts(x), verts(y)
    return float(cost_matrix(hx, hy, 1.0).max())


# --------------------------------------------------------------------------------------------
# Solve loop with periodic certificates (Algorithm 1 + best-so-far bounds, App. G.3)
# --------------------------------------------------------------------------------------------

def solve(r, c, C, eta, lam, max_iters, cert_every, omega, tol_abs=0.0, tol_rel=0.0,
          state: Optional[DualState] = None) -> dict:
    """Run Algorithm 1, evaluating the certificate every ``cert_every`` iterations.

    Best-so-far bounds U_best = min U_t, L_best = max L_t (App. G.3); stop when
    U_best - L_best <= tol_abs or (U_best - L_best)/U_best <= tol_rel.  The retained
    iterate is the certificate iteration with the lowest relative gap (U_t - L_t)/U_t
    (App. G, colour transfer).  Returns the history of (k, U, L) as well.
    """
    st = DualState.initial(len(r), len(c)) if state is None else state
    log_r, log_c = np.log(r), np.log(c)
    hist = []
    U_best, L_best = math.inf, -math.inf
    best = None
    stop = "max_iters"
    while st.k < max_iters:
        st = dual_obdrs_step(st, log_r, log_c, C, eta, lam)
        if cert_every > 0 and (st.k % cert_every == 0 or st.k == max_iters):
            cert = certificate_of(st, r, c, C, omega)
            hist.append((st.k, cert["U"], cert["L"]))
            U_best = min(U_best, cert["U"])
            L_best = max(L_best, cert["L"])
            rel = (cert["U"] - cert["L"]) / cert["U"]
            if best is None or rel < best["rel"]:
                best = dict(rel=rel, k=st.k, f=cert["f"], g=cert["g"], U=cert["U"], L=cert["L"])
            gap = U_best - L_best
            if (tol_abs > 0 and gap <= tol_abs) or (tol_rel > 0 and gap <= tol_rel * U_best):
                stop = "tol"
                break
    return dict(state=st, history=hist, U_best=U_best, L_best=L_best, best=best, stop=stop)


# --------------------------------------------------------------------------------------------
# Large instances: sampled rows, costs on the fly
# --------------------------------------------------------------------------------------------

def row_lse_sampled(rows, x, y, log_col, kappa, eps, chunk=1 << 16) -> np.ndarray:
    """LSE_j(log_col_j - C_ij/eps) for the listed rows i, over all columns, FP64.

    The cost is formed on the fly in column chunks so that no n x m matrix exists;
    used for spot checks where the dense oracle cannot run (Algorithm 1 row update).
    """
    x = np.asarray(x, np.float64)
    y = np.asarray(y, np.float64)
    log_col = np.asarray(log_col, np.float64)
    out = np.empty(len(rows))
    for t, i in enumerate(rows):
        parts = []
        for j0 in range(0, y.shape[0], chunk):
            yy = y[j0:j0 + chunk]
            Ci = kappa * ((yy - x[i][None, :]) ** 2).sum(axis=1)
            parts.append(log_col[j0:j0 + chunk] - Ci / eps)
        out[t] = lse(np.concatenate(parts), axis=0)
    return out


# --------------------------------------------------------------------------------------------
# Output of the colour-transfer application: barycentric projection, marginal errors
# --------------------------------------------------------------------------------------------

def plan_log(log_u, log_v, C, eps) -> np.ndarray:
    """log X_ij = log u_i + log v_j - C_ij / eps: the implicit plan diag(u) K diag(v), K = exp(-C/eps)."""
    return np.asarray(log_u, np.float64)[:, None] + np.asarray(log_v, np.float64)[None, :] - C / eps


def plan_diagnostics(log_u, log_v, C, eps, y, r, c) -> dict:
    """Barycentric projection and marginal errors of X = diag(u) K diag(v).

    Following App. G ("Implicit implementation and output"): the transferred colour of source
    point i is  y-hat_i = (sum_j X_ij y_j) / (sum_j X_ij).  The marginal errors of Tables 3 and 4
    compare the row sums of X with r and its column sums with c: the l1 error, the maximum absolute
    error and the maximum error relative to the prescribed mass.  Row and column sums are formed as
    exp(LSE) of the log-plan; the projection weights are the row-normalised plan.
    """
    LX = plan_log(log_u, log_v, C, eps)
    log_row = lse(LX, axis=1)
    log_col = lse(LX, axis=0)
    W = np.exp(LX - log_row[:, None])          # row-normalised plan
    y_hat = W @ np.asarray(y, np.float64)
    row = np.exp(log_row)
    col = np.exp(log_col)
    r = np.asarray(r, np.float64)
    c = np.asarray(c, np.float64)
    return {"y_hat": y_hat, "row_sums": row, "col_sums": col,
            "row_l1": float(np.abs(row - r).sum()), "row_max_abs": float(np.abs(row - r).max()),
            "row_max_rel": float((np.abs(row - r) / r).max()),
            "col_l1": float(np.abs(col - c).sum()), "col_max_abs": float(np.abs(col - c).max()),
            "col_max_rel": float((np.abs(col - c) / c).max())}


def projection_sampled(rows, x, y, log_u, log_v, kappa, eps, chunk=1 << 16):
    """(log row sum, y-hat) of X = diag(u) K diag(v) for the listed rows, costs formed on the fly."""
    x = np.asarray(x, np.float64)
    y = np.asarray(y, np.float64)
    log_v = np.asarray(log_v, np.float64)
    log_rows = np.empty(len(rows))
    y_hat = np.empty((len(rows), y.shape[1]))
    for t, i in enumerate(rows):
        parts = []
        for j0 in range(0, y.shape[0], chunk):
            yy = y[j0:j0 + chunk]
            Ci = kappa * ((yy - x[i][None, :]) ** 2).sum(axis=1)
            parts.append(log_v[j0:j0 + chunk] - Ci / eps)
        z = np.concatenate(parts)
        m = lse(z, axis=0)
        w = np.exp(z - m)
        log_rows[t] = float(log_u[i]) + m
        y_hat[t] = w @ y
    return log_rows, y_hat


def round_plan(log_u, log_v, C, eps, r, c) -> dict:
    """Round X = diag(u) K diag(v) onto Pi(r, c) (App. G "Momentum and Kernel Ablation" uses this to
    evaluate f, the cost of a feasible plan): scale the rows down to at most r, then the columns down
    to at most c, then add the rank-one correction err_r err_c^T / ||err_r||_1.  Returns the rounded
    plan, its cost <C, Z> and the cost of X before rounding, dense FP64."""
    X = np.exp(plan_log(log_u, log_v, C, eps))
    r = np.asarray(r, np.float64)
    c = np.asarray(c, np.float64)
    X1 = X * np.minimum(r / X.sum(axis=1), 1.0)[:, None]
    X2 = X1 * np.minimum(c / X1.sum(axis=0), 1.0)[None, :]
    er = r - X2.sum(axis=1)
    ec = c - X2.sum(axis=0)
    l1 = np.abs(er).sum()
    Z = X2 + (np.outer(er, ec) / l1 if l1 > 0 else 0.0)
    return {"Z": Z, "cost": float((C * Z).sum()), "cost_unrounded": float((C * X).sum()),
            "cost_scaled": float((C * X2).sum()), "err_r": er, "err_c": ec}
