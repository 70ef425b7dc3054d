"""The FP32 sweep's exp2 methods on the GPU against FP64 exp2.

The polynomial of OT_EXP_POLY / OT_EXP_SPLIT splits x = n + f with n = round(x) (exact) and
approximates 2^f on [-1/2, 1/2] by a degree-5 minimax polynomial (Remez fit by
csrc/fit_exp2_poly.py, max relative error 5.05e-7 in float32 Horner evaluation).  It is checked
over the whole range the sweeps feed it (x - shift in [-125, 126]) for its maximum relative error,
its mean (bias) and its exactness at integers, beside the SFU's ex2.approx for reference.
"""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu
P = pytest.importorskip("paper_2609_33814_b300")


def _inputs():
    rng = np.random.default_rng(7)
    grid = np.linspace(-125.0, 126.0, 1 << 20).astype(np.float32)
    near0 = rng.uniform(-1.0, 1.0, 1 << 18).astype(np.float32)
    halves = (np.arange(-125, 126) + 0.5).astype(np.float32)  # round-half boundaries of the split
    return np.concatenate([grid, near0, halves])


def test_polynomial_exp2_accuracy_and_bias():
    x = _inputs()
    ref = np.exp2(x.astype(np.float64))
    poly = P.probe_exp2(x, "poly").astype(np.float64)
    mufu = P.probe_exp2(x, "mufu").astype(np.float64)
    rel_p = (poly - ref) / ref
    rel_m = (mufu - ref) / ref
    assert np.abs(rel_p).max() <= 8e-7, np.abs(rel_p).max()      # fit 5.05e-7 + final rounding
    assert abs(rel_p.mean()) <= 5e-8, rel_p.mean()                # no systematic bias
    assert np.abs(rel_m).max() <= 4e-7                            # SFU reference (a few ulp)
    ints = np.arange(-125, 127).astype(np.float32)
    assert np.array_equal(P.probe_exp2(ints, "poly"), np.exp2(ints))  # 2^n exactly


def test_polynomial_exp2_clamps_out_of_range():
    x = np.array([-200.0, -126.5, 127.0, 300.0], np.float32)
    y = P.probe_exp2(x, "poly")
    assert np.all(np.isfinite(y)) and y[0] == y[1] == np.float32(2.0 ** -125)
    assert y[2] == y[3] == np.float32(2.0 ** 126)
