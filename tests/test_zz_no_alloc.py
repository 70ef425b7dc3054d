"""The allocation-free row update against the existing row update of ot_step.

``ot_row_update_noalloc`` is for callers that may not allocate device memory (a host runtime or
plugin that owns every device allocation); it keeps its working buffers in a fixed scratch array
inside the library.  Called twice in a row through the C ABI, on different inputs, each output
must match the row update that ``ot_step`` computes for the same state, within the FP32-sweep
tolerance used by the other parity tests (1e-5 relative in cost units).
"""
import ctypes as C

import numpy as np
import pytest

import ot_inputs as I

pytestmark = pytest.mark.gpu
P = pytest.importorskip("paper_2609_33814_b300")
torch = pytest.importorskip("torch")

TOL = 1e-5


def _lib():
    lib = P.lib()
    f = lib.ot_row_update_noalloc
    f.argtypes = [C.c_int64, C.c_int64, C.c_int32, C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p, C.c_double,
                  C.c_double, C.c_void_p, C.c_uint64]
    f.restype = C.c_int
    return f


def _reference(ctx, prob, log_bt, eps):
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
    r = I.Problem(x, y, I.uniform_weights(3000, 10), I.uniform_weights(2000, 11), 1.0 / 3.0, 1.0, "ragged3")
    return [(g, 0.05), (r, 0.02)]


def test_noalloc_row_update_matches_step_twice():
    fn = _lib()
    ctx = P.Context(0)
    rng = np.random.default_rng(3)
    for prob, eps in _cases():
        dx = torch.from_numpy(prob.x).cuda()
        dy = torch.from_numpy(prob.y).cuda()
        a = prob.a / prob.a.sum()
        dlr = torch.from_numpy(np.log(a)).cuda()
        for call in range(2):  # two calls in a row share the scratch array
            log_bt = rng.normal(0.0, 3.0, prob.m) / eps * 0.01
            ref = _reference(ctx, prob, log_bt, eps)
            dbt = torch.from_numpy(log_bt).cuda()
            out = torch.full((prob.n,), float("nan"), dtype=torch.float64, device="cuda")
            torch.cuda.synchronize()
            st = fn(prob.n, prob.m, prob.d, dx.data_ptr(), dy.data_ptr(), dlr.data_ptr(), dbt.data_ptr(),
                    prob.kappa, eps, out.data_ptr(), 0)
            assert st == P.OT_OK, (prob.name, call, st)
            got = out.cpu().numpy()
            err = np.abs(eps * (got - ref)).max() / np.abs(eps * ref).max()
            assert err <= TOL, (prob.name, call, err)
    ctx.close()


def test_noalloc_rejects_sizes_beyond_its_scratch():
    fn = _lib()
    n = 16385
    x = torch.zeros((n, 2), dtype=torch.float32, device="cuda")
    lr = torch.zeros(n, dtype=torch.float64, device="cuda")
    out = torch.zeros(n, dtype=torch.float64, device="cuda")
    st = fn(n, 4, 2, x.data_ptr(), x.data_ptr(), lr.data_ptr(), lr.data_ptr(), 1.0, 1.0, out.data_ptr(), 0)
    assert st == P.OT_EINVAL
