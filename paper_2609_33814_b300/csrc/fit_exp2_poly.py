"""Fit the polynomial of the FMA-pipe exp2 used by the FP32 sweep and write ``ot_exp2_poly.cuh``.

Method: 2^x = 2^n * 2^f with n = round(x) and f = x - n in [-1/2, 1/2]; 2^f is approximated
by a degree-``DEG`` polynomial whose coefficients minimise the maximum *relative* error on
[-1/2, 1/2] (Remez exchange on the equioscillation points, started from a least-squares fit
on Chebyshev nodes).  The constant term is pinned to 1 so that 2^0 = 1 exactly.  The
coefficients are then rounded to float32 and the error of the rounded polynomial, evaluated
by Horner's rule in float32, is reported.

Run: ``python fit_exp2_poly.py`` (rewrites the header next to this script).
"""
import os

import numpy as np

DEG = 5


def _fit(deg: int, iters: int = 30):
    # unknowns c1..c_deg and the levelled error E: p(f) = 1 + sum c_k f^k, (p - 2^f)/2^f = +-E
    k = np.arange(deg + 2)
    pts = 0.5 * np.cos(np.pi * k / (deg + 1))[::-1]  # deg+2 alternation points
    for _ in range(iters):
        A = np.zeros((deg + 1, deg + 1))
        rhs = np.zeros(deg + 1)
        # use deg+1 of the points (constant fixed to 1 removes one unknown)
        use = pts[: deg + 1] if len(pts) > deg + 1 else pts
        for i, f in enumerate(use):
            t = 2.0 ** f
            A[i, :deg] = [f ** j for j in range(1, deg + 1)]
            A[i, deg] = -((-1) ** i) * t
            rhs[i] = t - 1.0
        sol = np.linalg.solve(A, rhs)
        c = np.concatenate([[1.0], sol[:deg]])
        grid = np.linspace(-0.5, 0.5, 200001)
        err = (np.polyval(c[::-1], grid) - 2.0 ** grid) / 2.0 ** grid
        # new alternation points: extrema of err between sign changes
        sign = np.sign(err)
        idx = np.where(np.diff(sign) != 0)[0]
        bounds = np.concatenate([[0], idx + 1, [len(grid)]])
        ext = [b0 + int(np.argmax(np.abs(err[b0:b1]))) for b0, b1 in zip(bounds[:-1], bounds[1:]) if b1 > b0]
        if len(ext) >= deg + 1:
            ext = sorted(ext, key=lambda i: -abs(err[i]))[: deg + 1]
            pts = np.sort(grid[ext])
    return c


def main():
    c = _fit(DEG)
    c32 = c.astype(np.float32)
    f = np.linspace(-0.5, 0.5, 400001).astype(np.float32)
    p = np.full_like(f, c32[DEG])
    for j in range(DEG - 1, -1, -1):
        p = (p * f + c32[j]).astype(np.float32)
    rel = np.abs(p.astype(np.float64) - 2.0 ** f.astype(np.float64)) / 2.0 ** f.astype(np.float64)
    print(f"degree {DEG}: max relative error (float32 Horner) = {rel.max():.3e}")
    lines = [
        "// Generated by fit_exp2_poly.py: minimax (relative error) polynomial for 2^f on [-1/2, 1/2],",
        f"// degree {DEG}, constant term 1; max relative error of the float32 Horner evaluation {rel.max():.3e}.",
        "#pragma once",
        "namespace ot {",
        f"constexpr int kExp2PolyDeg = {DEG};",
        "__device__ constexpr float kExp2Poly[kExp2PolyDeg + 1] = {"
        + ", ".join(f"{float(v)!r}f" for v in c32) + "};",
        "}  // namespace ot",
        "",
    ]
    out = os.path.join(os.path.dirname(os.path.abspath(__file__)), "ot_exp2_poly.cuh")
    open(out, "w").write("\n".join(lines))
    print("wrote", out)


if __name__ == "__main__":
    main()
