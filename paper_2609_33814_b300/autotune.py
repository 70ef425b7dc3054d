"""Tile-plan autotuner: times every instantiated sweep kernel (points per thread R, chunk width CH)
for each point dimension d and precision mode on this GPU, and writes the fastest as the plan table
``tile_plans.txt`` that the library reads beside ``libot.so`` when its first context is created.

Run on the GPU the library will serve on::

    python paper_2609_33814_b300/autotune.py [--out PATH] [--seconds 0.3]

Each candidate runs a representative resident instance (d = 1: 2^17 points on a line, d = 2: a
256 x 256 grid, d = 3: 2^18 RGB colours; a quarter of the points for FP64) past its first iterations,
so that the sweeps' shift hints are active, and is timed over whole iterations (both sweeps).  The
table's lines are ``d precision R CH`` with the ot_precision values of ``include/ot.h``; the measured
rates are written beside them as comments.  A plan changes results bitwise (summation order), never
their accuracy; the built-in plans are the choices of this script on B300.
"""
from __future__ import annotations

import argparse
import datetime
import os
import sys
import time

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.dirname(_HERE))

import ot_inputs as I  # noqa: E402
import paper_2609_33814_b300 as P  # noqa: E402

CANDIDATES = {
    "mufu": [(1, 8), (1, 16), (2, 8), (2, 16), (4, 8), (4, 16), (8, 8)],
    "poly": [(2, 16), (4, 16)],
    "split": [(2, 16), (4, 16)],
    "comp": [(1, 8), (2, 8), (4, 8)],
    "fp64": [(1, 8), (2, 8)],
}


def problem(d: int, small: bool):
    if d == 1:
        n = (1 << 15) if small else (1 << 17)
        x = I.random_cloud(n, 1, 7)
        y = I.random_cloud(n, 1, 8)
        return I.Problem(x, y, I.uniform_weights(n, 9), I.uniform_weights(n, 10), 1.0, 1.0, "line")
    if d == 2:
        return I.grid_problem(64 if small else 256, 11, "gaussmix", "cauchy")
    return I.rgb_problem((1 << 14) if small else (1 << 18), 12)


def rate(ctx, prob, precision: str, seconds: float) -> float:
    """Implicit entries/s of whole iterations of one resident instance."""
    import torch
    S = ctx.state(prob.x, prob.y, prob.a, prob.b, cost_scale=prob.kappa, omega=prob.omega, eps0=1.0, lam=1.0,
                  precision=precision, cert_every=0)
    S.step(3)  # past k = 2: shift hints active
    torch.cuda.synchronize()
    t = time.perf_counter()
    S.step(1)
    torch.cuda.synchronize()
    per = max(time.perf_counter() - t, 1e-6)
    iters = max(1, int(seconds / per))
    t = time.perf_counter()
    S.step(iters)
    torch.cuda.synchronize()
    dt = time.perf_counter() - t
    S.close()
    return 2.0 * prob.n * prob.m * iters / dt


def main() -> None:
    ap = argparse.ArgumentParser(description=__doc__.splitlines()[0])
    ap.add_argument("--out", default=os.path.join(_HERE, "tile_plans.txt"))
    ap.add_argument("--seconds", type=float, default=0.3, help="timed work per candidate")
    ap.add_argument("--precisions", default="mufu,poly,split,comp,fp64")
    args = ap.parse_args()
    import torch
    ctx = P.Context(0)
    lines = [f"# tile plans measured by autotune.py on {torch.cuda.get_device_name(0)}, "
             f"{datetime.datetime.now(datetime.timezone.utc).strftime('%Y-%m-%d %H:%M UTC')}",
             "# d precision R CH   (precision: 0 mufu, 1 poly, 2 split, 3 fp64, 4 comp)"]
    for d in (1, 2, 3):
        for precision in args.precisions.split(","):
            prob = problem(d, small=precision == "fp64")
            results = []
            for R, ch in CANDIDATES[precision]:
                P.set_tile_plan(d, precision, R, ch)
                results.append((rate(ctx, prob, precision, args.seconds), R, ch))
            P.set_tile_plan(d, precision, 0, 0)
            best = max(results)
            lines.append(f"{d} {P.PRECISIONS[precision]} {best[1]} {best[2]}   # {precision}: " +
                         ", ".join(f"R{R}/CH{ch} {v:.3e}" for v, R, ch in results) + " entries/s")
            print(lines[-1], flush=True)
    with open(args.out, "w") as f:
        f.write("\n".join(lines) + "\n")
    print("wrote", args.out)


if __name__ == "__main__":
    main()
