"""Continuous-batching server: every result is the same alone and in the mix.

An instance's work items (points per thread, chunk width, split counts) depend only on its own
sizes and precision, and every reduction runs in a fixed order, so a request solved inside a mixed
batch (uneven sizes, classes, lambda, lanes) must reproduce the same request solved alone by
``ot_solve`` bit for bit: iteration count, stop reason, certificate bounds and potentials.
"""
import threading

import numpy as np
import pytest

import ot_inputs as I

pytestmark = pytest.mark.gpu
P = pytest.importorskip("paper_2609_33814_b300")


@pytest.fixture(scope="module")
def ctx():
    return P.Context(0)


def _mix():
    out = []
    out.append((I.grid_problem(16, 1), dict(lam=1.0)))
    out.append((I.grid_problem(24, 2, "gaussmix", "cauchy"), dict(lam=1.5)))
    out.append((I.grid_problem(32, 3, "sparse", "uniform"), dict(lam=1.0)))
    x = I.random_cloud(300, 2, 4)
    y = I.random_cloud(200, 2, 5)
    out.append((I.Problem(x, y, I.uniform_weights(300, 6), I.uniform_weights(200, 7), 0.5, 1.0, "ragged"),
                dict(lam=1.99, eps0=0.5)))
    out.append((I.grid_problem(20, 8, "cauchy", "gaussmix"), dict(lam=1.2)))
    out.append((I.grid_problem(40, 9, "gaussmix", "gaussmix"), dict(lam=1.0)))
    return out


def _params(extra, **kw):
    p = dict(eps0=1.0, lam=1.0, max_iters=600, cert_every=100, precision="mufu", tol_rel=0.02)
    p.update(extra)
    p.update(kw)
    return p


def _same(solo, batched, what):
    f0, g0, r0 = solo
    f1, g1, r1 = batched
    assert r1["iters"] == r0["iters"], (what, r0["iters"], r1["iters"])
    assert r1["stop"] == r0["stop"], what
    assert r1["best_iter"] == r0["best_iter"], what
    assert r1["U_best"] == r0["U_best"] and r1["L_best"] == r0["L_best"], (what, r0, r1)
    scale = max(np.abs(f0).max(), np.abs(g0).max())
    err = max(np.abs(f1 - f0).max(), np.abs(g1 - g0).max()) / scale
    assert np.array_equal(f1, f0) and np.array_equal(g1, g0), (what, err)


def test_each_result_same_alone_and_in_mix(ctx):
    mix = _mix()
    solo = [ctx.solve(p.x, p.y, p.a, p.b, cost_scale=p.kappa, omega=p.omega, zero_mass_floor=1e-15,
                      **_params(extra)) for p, extra in mix]
    srv = P.Server(ctx, hbm_budget_bytes=4 << 30, max_slots=16)
    ids = [srv.submit(p.x, p.y, p.a, p.b, cost_scale=p.kappa, omega=p.omega, zero_mass_floor=1e-15,
                      **_params(extra)) for p, extra in mix]
    outs = [srv.wait(i, 120.0) for i in ids]
    for (p, _), s, b in zip(mix, solo, outs):
        _same(s, b, p.name)
    st = srv.stats()
    assert st["completed"] == len(mix) and st["failed"] == 0
    assert st["p99_latency_s"] >= st["p50_latency_s"] > 0
    srv.close()


def test_mixed_lanes_d3_and_fp64(ctx):
    rgb = I.rgb_problem(500, seed=11, m=400)
    grid = I.grid_problem(16, 12, "gaussmix", "uniform")
    reqs = [(rgb, _params({}, eps0=0.1, max_iters=300, tol_rel=0.0)),
            (grid, _params({}, precision="fp64", max_iters=300, tol_rel=0.0)),
            (grid, _params({}, max_iters=300, tol_rel=0.0))]
    solo = [ctx.solve(p.x, p.y, p.a, p.b, cost_scale=p.kappa, omega=p.omega, **kw) for p, kw in reqs]
    srv = P.Server(ctx, hbm_budget_bytes=1 << 30, max_slots=8)
    ids = [srv.submit(p.x, p.y, p.a, p.b, cost_scale=p.kappa, omega=p.omega, **kw) for p, kw in reqs]
    for (p, kw), s, i in zip(reqs, solo, ids):
        _same(s, srv.wait(i, 120.0), f"{p.name}/{kw['precision']}")
    srv.close()


def test_budget_slots_and_oversized_request(ctx):
    p = I.grid_problem(16, 3)
    srv = P.Server(ctx, hbm_budget_bytes=1 << 20, max_slots=2)
    ids = [srv.submit(p.x, p.y, p.a, p.b, cost_scale=p.kappa, omega=p.omega, **_params({}, max_iters=200))
           for _ in range(5)]
    for i in ids:
        f, g, r = srv.wait(i, 120.0)
        assert r["iters"] == 200 and r["queue_s"] >= 0.0
    big = I.grid_problem(64, 4)
    with pytest.raises(P.OTError) as e:
        srv.submit(big.x, big.y, big.a, big.b, cost_scale=big.kappa, omega=big.omega, **_params({}))
    assert e.value.status == P.OT_ENOMEM
    assert srv.stats()["completed"] == 5
    srv.close()


def test_cancel(ctx):
    p = I.grid_problem(32, 5)
    srv = P.Server(ctx, hbm_budget_bytes=1 << 30, max_slots=4)
    rid = srv.submit(p.x, p.y, p.a, p.b, cost_scale=p.kappa, omega=p.omega,
                     **_params({}, max_iters=10 ** 7, tol_rel=0.0))
    assert srv.poll(rid) is None
    srv.cancel(rid)
    with pytest.raises(P.OTError) as e:
        srv.wait(rid, 60.0)
    assert e.value.status == P.OT_ECANCELLED
    assert srv.stats()["cancelled"] == 1
    srv.close()


def test_concurrent_submitters_device_inputs(ctx):
    """Four host threads submit device-resident requests at once; each result is bitwise the same
    request solved alone by ot_solve."""
    import torch
    srv = P.Server(ctx, hbm_budget_bytes=2 << 30, max_slots=32)
    results = {}
    lock = threading.Lock()

    def worker(t):
        for j in range(4):
            p = I.grid_problem(12 + 4 * j, 100 * t + j, "gaussmix", "uniform")
            dev = [torch.from_numpy(v).cuda() for v in (p.x, p.y, p.a, p.b)]
            rid = srv.submit(*dev, cost_scale=p.kappa, omega=p.omega, **_params({}, max_iters=300))
            with lock:
                results[rid] = p

    ths = [threading.Thread(target=worker, args=(t,)) for t in range(4)]
    for t in ths:
        t.start()
    for t in ths:
        t.join()
    assert len(results) == 16
    for rid, p in results.items():
        batched = srv.wait(rid, 120.0)
        solo = ctx.solve(p.x, p.y, p.a, p.b, cost_scale=p.kappa, omega=p.omega, **_params({}, max_iters=300))
        _same(solo, batched, p.name)
    srv.close()
