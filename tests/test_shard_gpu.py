"""Row-sharded execution on the GPU: two ranks (processes over gloo) each update a slice of the
points of one problem on the same device, exchanging packed operands after every half-sweep and
the certificate's partial sums on certificate iterations (``paper_2609_33814_b300.shard``).

Checks, per problem (a 48 x 48 grid pair at lambda = 1.5, and a ragged 1500 x 1300 RGB pair):
* after K iterations, the gathered potentials match an unsharded ``ot_state`` run of the same
  iterations within the FP32-sweep tolerance (1e-5 relative, cost units; the two differ only where a
  slice's shift hints are withdrawn while the whole side's are not), and the certificates within 1e-6;
* the next sharded iteration matches the oracle's iteration from the gathered state (Algorithm 1,
  one-step parity at 1e-5), and the last certificate matches the oracle's certificate (Prop. 3 with
  Algorithm 2) of the gathered state within 1e-6.
Kernels of the two ranks never wait for each other: all exchange runs on the host between launches.
"""
import os
import socket

import numpy as np
import pytest

pytestmark = pytest.mark.gpu
P = pytest.importorskip("paper_2609_33814_b300")
torch = pytest.importorskip("torch")

TOL_POT = 1e-5
TOL_CERT = 1e-6


def _problem(kind):
    import ot_inputs as I
    if kind == "grid48":
        return I.grid_problem(48, 17, "gaussmix", "cauchy"), dict(eps0=1.0, lam=1.5)
    x = I.random_cloud(1500, 3, 5)
    y = I.random_cloud(1300, 3, 6)
    return (I.Problem(x, y, I.uniform_weights(1500, 7), I.uniform_weights(1300, 8), 1.0 / 3.0, 1.0, "rgb_ragged"),
            dict(eps0=0.1, lam=1.0))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, kind, iters, ce, q):
    import torch.distributed as td
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    td.init_process_group("gloo", rank=rank, world_size=world)
    import paper_2609_33814_b300 as Pk
    from paper_2609_33814_b300 import shard
    prob, prm = _problem(kind)
    ctx = Pk.Context(0)
    st = Pk.ShardState(ctx, prob.x, prob.y, prob.a, prob.b, rank, world, cost_scale=prob.kappa, omega=prob.omega,
                       cert_every=ce, precision="mufu", **prm)
    res = shard.run(st, iters, ce, prob.omega)
    vec = {w: shard.gather_vector(st, w, 0 if w in (Pk.OT_LOG_ALPHA, Pk.OT_LOG_ALPHA_HAT) else 1)
           for w in (Pk.OT_LOG_ALPHA, Pk.OT_LOG_ALPHA_HAT, Pk.OT_LOG_BETA, Pk.OT_LOG_BETA_PREV, Pk.OT_LOG_BETA_HAT,
                     Pk.OT_LOG_BETA_TILDE)}
    # one more (certificate) iteration for the one-step comparison with the oracle
    nxt = shard.run(st, 1, 1, prob.omega, k0=iters)
    vec2 = {w: shard.gather_vector(st, w, 0 if w == Pk.OT_LOG_ALPHA_HAT else 1)
            for w in (Pk.OT_LOG_ALPHA_HAT, Pk.OT_LOG_BETA_HAT)}
    if rank == 0:
        q.put((res, vec, nxt, vec2))
    st.close()
    ctx.close()
    td.destroy_process_group()


@pytest.mark.parametrize("kind", ["grid48", "rgb_ragged"])
def test_two_rank_sharded_solve(kind):
    import oracle as O
    world, iters, ce = 2, 120, 40
    mpc = torch.multiprocessing.get_context("spawn")
    q = mpc.Queue()
    port = _free_port()
    procs = [mpc.Process(target=_worker, args=(r, world, port, kind, iters, ce, q)) for r in range(world)]
    for p in procs:
        p.start()
    res, vec, nxt, vec2 = q.get(timeout=600)
    for p in procs:
        p.join(timeout=120)
        assert p.exitcode == 0
    prob, prm = _problem(kind)
    a = prob.a / prob.a.sum()
    b = prob.b / prob.b.sum()
    # against an unsharded run of the same iterations
    ctx = P.Context(0)
    S = ctx.state(prob.x, prob.y, prob.a, prob.b, cost_scale=prob.kappa, omega=prob.omega, cert_every=ce,
                  precision="mufu", **prm)
    r1 = S.step(iters)
    eps = O.eps_schedule(prm["eps0"], prm["lam"], iters - 1)
    lah, lbh = S.get(P.OT_LOG_ALPHA_HAT), S.get(P.OT_LOG_BETA_HAT)
    scale = max(np.abs(eps * lah).max(), np.abs(eps * (lbh - np.log(b))).max())
    err = max(np.abs(vec[P.OT_LOG_ALPHA_HAT] - lah).max(), np.abs(vec[P.OT_LOG_BETA_HAT] - lbh).max()) * eps / scale
    assert err <= TOL_POT, err
    assert abs(res["U_best"] - r1["U_best"]) <= TOL_CERT and abs(res["L_best"] - r1["L_best"]) <= TOL_CERT
    S.close()
    ctx.close()
    # the next iteration against the oracle's from the gathered state
    C_ = O.cost_matrix(prob.x, prob.y, prob.kappa)
    st = O.DualState(vec[P.OT_LOG_ALPHA], vec[P.OT_LOG_BETA], vec[P.OT_LOG_BETA_PREV], vec[P.OT_LOG_ALPHA_HAT],
                     vec[P.OT_LOG_BETA_HAT], vec[P.OT_LOG_BETA_TILDE], iters, eps)
    st1 = O.dual_obdrs_step(st, np.log(a), np.log(b), C_, prm["eps0"], prm["lam"])
    f_o, g_o = st1.eps * st1.log_alpha_hat, st1.eps * (st1.log_beta_hat - np.log(b))
    f_g, g_g = st1.eps * vec2[P.OT_LOG_ALPHA_HAT], st1.eps * (vec2[P.OT_LOG_BETA_HAT] - np.log(b))
    scale = max(np.abs(f_o).max(), np.abs(g_o).max())
    assert max(np.abs(f_g - f_o).max(), np.abs(g_g - g_o).max()) / scale <= TOL_POT
    # its certificate (the sharded one is a compensated certificate iteration)
    cert = O.certificate(vec2[P.OT_LOG_ALPHA_HAT], vec2[P.OT_LOG_BETA_HAT], st1.log_beta_tilde, a, b, C_, st1.eps,
                         prob.omega)
    (k, U, L), = nxt["certificates"]
    assert k == iters + 1
    assert abs(U - cert["U"]) <= TOL_CERT and abs(L - cert["L"]) <= TOL_CERT, (U, cert["U"], L, cert["L"])
