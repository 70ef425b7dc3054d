"""Row-sharded solve of one problem over the ranks of a ``torch.distributed`` process group.

Host orchestration of the library's slice states (``ot_shard_*`` in ``include/ot.h``): every rank
holds the whole problem's packed operands and updates its own slice of the points of each side.
After each half-sweep of Algorithm 1 (the row update, then the column update) the ranks allgather
the packed operands their slices rewrote, and on certificate iterations they allreduce the four
partial sums of Proposition 3: L = sum <r, f> + sum <c, g>, U = sum <t, w> + omega sum delta.  The
exchange runs on the host (gloo or NCCL over host tensors); no kernel waits for another rank.
"""
from __future__ import annotations

import numpy as np


def exchange(st, side: int, group=None):
    """Allgather the pack slices of ``side``: every rank's bytes go to every other rank's state.

    ``st`` is a slice state (``ShardState``, or any object with its ``rank``, ``world``,
    ``pack_bytes``, ``pack_get`` and ``pack_put``)."""
    import torch
    import torch.distributed as td
    sizes = [st.pack_bytes(side, r) for r in range(st.world)]
    top = max(sizes)
    mine = np.zeros(top, np.uint8)
    own = st.pack_get(side)
    mine[:own.size] = own
    bufs = [torch.zeros(top, dtype=torch.uint8) for _ in range(st.world)]
    td.all_gather(bufs, torch.from_numpy(mine), group=group)
    for r in range(st.world):
        if r != st.rank:
            st.pack_put(side, r, bufs[r].numpy()[:sizes[r]])


def certificate(st, omega: float, group=None):
    """(U, L, eps) of the certificate iteration just completed, summed over the ranks."""
    import torch
    import torch.distributed as td
    p = st.cert_partials()
    t = torch.tensor(p[:4], dtype=torch.float64)
    td.all_reduce(t, group=group)
    rf, cg, tw, delta = (float(v) for v in t)
    return tw + omega * delta, rf + cg, float(p[4])


def run(st, iters: int, cert_every: int, omega: float, group=None, k0: int = 0):
    """``iters`` iterations of Algorithm 1 on the slice states of the group, from iteration k0.
    Returns the certificates [(k, U, L)] and the best-so-far bounds (App. G.3)."""
    certs = []
    for k in range(k0, k0 + iters):
        cert = cert_every > 0 and (k + 1) % cert_every == 0
        for side in (0, 1):
            st.half_sweep(side, cert)
            exchange(st, side, group)
        if cert:
            U, L, _ = certificate(st, omega, group)
            certs.append((k + 1, U, L))
    U_best = min((c[1] for c in certs), default=float("inf"))
    L_best = max((c[2] for c in certs), default=float("-inf"))
    return {"certificates": certs, "U_best": U_best, "L_best": L_best}


def gather_vector(st, which: int, side: int, group=None) -> np.ndarray:
    """A whole state vector of ``side`` (0: n entries, 1: m) assembled from every rank's slice."""
    import torch
    import torch.distributed as td
    v = st.get(which)
    own = np.zeros_like(v)
    p0, p1 = st.slice(side)
    own[p0:p1] = v[p0:p1]
    t = torch.from_numpy(own)
    td.all_reduce(t, group=group)
    return t.numpy()
