"""Study of the fast sweep's FP32 exponent under gauge drift (not a test; run by hand).

Runs Dual O-BDRS (Algorithm 1) on one grid pair three ways and prints the certified relative gap
(Prop. 3, computed in FP64 from each run's own iterates) every 1000 iterations:
  fp64   the oracle's iteration;
  nooff  the log-sum-exps with the fast sweep's FP32 exponent: h_q = (lv_q - kappa|w_q|^2/eps) log2 e
         rounded to FP32, A_p = (2 kappa log2 e / eps) u_p rounded to FP32, z = h_q + <A_p, w_q> in
         FP32, the sum and the rest in FP64;
  off    the same with h_q - G stored instead of h_q (G = h_0), G added back in FP64.
With --center the FP32 runs translate both clouds by the grid's centre ((s - 1)/2 per axis, exact
for integer coordinates), which leaves the cost unchanged and shrinks |h| and |<A, w>| about 4x.

    python tests/fp32_exponent_study.py --mode off --size 16 --iters 30000 --lam 1.99
"""
import argparse
import os
import sys

import numpy as np

sys.path.insert(0, os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
import oracle as O  # noqa: E402
import ot_inputs as I  # noqa: E402

LOG2E = 1.4426950408889634
LN2 = 0.6931471805599453


def lse_fp32(lv, U, W, wn2, un2, kappa, eps, offset):
    """LSE_q(lv_q - kappa |u_p - w_q|^2 / eps) per point p of U, with an FP32 exponent."""
    h = (lv - wn2 / eps) * LOG2E
    G = h[0] if offset else 0.0
    h32 = (h - G).astype(np.float32)
    A32 = (2.0 * kappa * LOG2E / eps * U).astype(np.float32)
    z = (h32[None, :] + (A32 @ W.astype(np.float32).T).astype(np.float32)).astype(np.float64)
    m = z.max(1)
    return (m + np.log2(np.exp2(z - m[:, None]).sum(1)) + G) * LN2 - un2 / eps


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--mode", choices=["fp64", "nooff", "off"], default="off")
    ap.add_argument("--size", type=int, default=16)
    ap.add_argument("--iters", type=int, default=30000)
    ap.add_argument("--lam", type=float, default=1.99)
    ap.add_argument("--seed", type=int, default=91)
    ap.add_argument("--center", action="store_true")
    args = ap.parse_args()
    p = I.grid_problem(args.size, args.seed, "cauchy", "gaussmix")
    a = np.maximum(p.a, 1e-15)
    a = a / a.sum()
    b = np.maximum(p.b, 1e-15)
    b = b / b.sum()
    C = O.cost_matrix(p.x, p.y, p.kappa)
    X, Y = p.x.astype(np.float64), p.y.astype(np.float64)
    if args.center:
        X, Y = X - (args.size - 1) / 2.0, Y - (args.size - 1) / 2.0
    xn2, yn2 = p.kappa * (X ** 2).sum(1), p.kappa * (Y ** 2).sum(1)
    la, lb, lam = np.log(a), np.log(b), args.lam
    st = O.DualState.initial(p.n, p.m)
    U_best, L_best = np.inf, -np.inf
    for k in range(1, args.iters + 1):
        eps = O.eps_schedule(1.0, lam, st.k)
        bt = st.log_beta + (st.log_beta - st.log_beta_prev) / lam
        if args.mode == "fp64":
            lah = la - O.lse(bt[None, :] - C / eps, axis=1)
        else:
            lah = la - lse_fp32(bt, X, Y, yn2, xn2, p.kappa, eps, args.mode == "off")
        if args.mode == "fp64":
            lbh = lb - O.lse(lah[:, None] - C / eps, axis=0)
        else:
            lbh = lb - lse_fp32(lah, Y, X, xn2, yn2, p.kappa, eps, args.mode == "off")
        st = O.DualState((1 - lam) * st.log_alpha + lam * lah, (1 - lam) * st.log_beta + lam * lbh, st.log_beta,
                         lah, lbh, bt, st.k + 1, eps)
        if k % 1000 == 0:
            c = O.certificate_of(st, a, b, C, 1.0)
            U_best, L_best = min(U_best, c["U"]), max(L_best, c["L"])
            print(f"{args.mode} k={k} eps={eps:.2e} rel_gap={(U_best - L_best) / U_best:.3e} "
                  f"max|log beta|={np.abs(st.log_beta).max():.3e}", flush=True)


if __name__ == "__main__":
    main()
