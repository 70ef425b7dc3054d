"""Python binding of the B300 Dual (O-)BDRS optimal-transport solver.

A thin ctypes layer over the C ABI in ``include/ot.h`` (``libot.so``, built in-tree by
``paper_2609_33814_b300.build``): argument marshalling only.  Every step of the solver
runs in the library's CUDA kernels; there is no CPU fallback, and importing the
package fails loudly when the shared library is missing.

Inputs may be numpy arrays (host) or CUDA torch tensors (device pointers are passed
through, ``on_device = 1``).  Point clouds are float32 ``(n, d)``, weights float64.
"""
from __future__ import annotations

import ctypes as C
import os
from dataclasses import dataclass
from typing import Optional

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libot.so")

if not os.path.exists(LIB_PATH):
    raise ImportError(
        f"{LIB_PATH} is missing: build it with `python paper_2609_33814_b300/build.py` "
        "(the solver has no CPU fallback)")

_lib = C.CDLL(LIB_PATH)

# --- enums (mirror include/ot.h) ----------------------------------------------------------
OT_OK, OT_EINVAL, OT_ENOMEM, OT_ECUDA, OT_ENUMERIC, OT_ETIMEDOUT, OT_EBUSY, OT_ECANCELLED, OT_ENOTFOUND = range(9)
OT_EXP_MUFU, OT_EXP_POLY, OT_EXP_SPLIT, OT_FP64, OT_FP32_COMP = range(5)
OT_STOP_TOL, OT_STOP_MAX_ITERS, OT_STOP_TIME, OT_STOP_NONE = range(4)
(OT_LOG_ALPHA, OT_LOG_ALPHA_HAT, OT_LOG_BETA, OT_LOG_BETA_PREV, OT_LOG_BETA_HAT, OT_LOG_BETA_TILDE,
 OT_F_CERT, OT_G_CERT, OT_F_BEST, OT_G_BEST) = range(10)

PRECISIONS = {"mufu": OT_EXP_MUFU, "poly": OT_EXP_POLY, "split": OT_EXP_SPLIT, "fp64": OT_FP64,
              "comp": OT_FP32_COMP}
STOP_NAMES = {OT_STOP_TOL: "tol", OT_STOP_MAX_ITERS: "max_iters", OT_STOP_TIME: "time", OT_STOP_NONE: "none"}


class OtProblem(C.Structure):
    _fields_ = [("n", C.c_int64), ("m", C.c_int64), ("d", C.c_int32), ("on_device", C.c_int32),
                ("x", C.c_void_p), ("y", C.c_void_p), ("a", C.c_void_p), ("b", C.c_void_p),
                ("cost_scale", C.c_double), ("omega", C.c_double), ("zero_mass_floor", C.c_double)]


class OtParams(C.Structure):
    _fields_ = [("eps0", C.c_double), ("lam", C.c_double), ("max_iters", C.c_int64),
                ("time_budget_s", C.c_double), ("cert_every", C.c_int32), ("precision", C.c_int32),
                ("tol_abs", C.c_double), ("tol_rel", C.c_double), ("stream", C.c_uint64),
                ("algorithm", C.c_int32), ("refine_on", C.c_double), ("refine_tol", C.c_double)]


ALGORITHMS = {"bdrs": 0, "as": 1, "as_momentum": 2, "as_current": 3, "das": 4}


class OtResult(C.Structure):
    _fields_ = [("iters", C.c_int64), ("best_iter", C.c_int64), ("n_certs", C.c_int64),
                ("U", C.c_double), ("L", C.c_double), ("U_best", C.c_double), ("L_best", C.c_double),
                ("gap_abs", C.c_double), ("gap_rel", C.c_double), ("eps_final", C.c_double),
                ("elapsed_s", C.c_double), ("kappa", C.c_double), ("omega", C.c_double),
                ("stop", C.c_int32), ("device_errors", C.c_int32), ("latency_s", C.c_double),
                ("queue_s", C.c_double)]

    def as_dict(self) -> dict:
        d = {f: getattr(self, f) for f, _ in self._fields_}
        d["stop"] = STOP_NAMES.get(self.stop, self.stop)
        return d


class OtServeStats(C.Structure):
    _fields_ = [("submitted", C.c_int64), ("completed", C.c_int64), ("cancelled", C.c_int64),
                ("failed", C.c_int64), ("active", C.c_int64), ("pending", C.c_int64), ("chunks", C.c_int64),
                ("launches", C.c_int64), ("p50_latency_s", C.c_double), ("p99_latency_s", C.c_double),
                ("mean_latency_s", C.c_double), ("solves_per_s", C.c_double), ("entries_per_s", C.c_double),
                ("entries", C.c_double), ("elapsed_s", C.c_double), ("hbm_used_bytes", C.c_double)]

    def as_dict(self) -> dict:
        return {f: getattr(self, f) for f, _ in self._fields_}


_P = C.c_void_p
_lib.ot_params_default.argtypes = [C.POINTER(OtParams)]
_lib.ot_status_str.restype = C.c_char_p
_lib.ot_status_str.argtypes = [C.c_int]
_lib.ot_last_error.restype = C.c_char_p
_lib.ot_last_error.argtypes = [_P]
_lib.ot_context_create.argtypes = [C.c_int, C.POINTER(_P)]
_lib.ot_context_destroy.argtypes = [_P]
_lib.ot_solve.argtypes = [_P, C.POINTER(OtProblem), C.POINTER(OtParams), _P, _P, C.POINTER(OtResult)]
_lib.ot_state_create.argtypes = [_P, C.POINTER(OtProblem), C.POINTER(OtParams), C.POINTER(_P)]
_lib.ot_state_destroy.argtypes = [_P]
_lib.ot_step.argtypes = [_P, C.c_int64, C.POINTER(OtResult)]
_lib.ot_certificate.argtypes = [_P, C.POINTER(OtResult)]
_lib.ot_state_get.argtypes = [_P, C.c_int, _P, C.POINTER(C.c_int64)]
_lib.ot_state_set.argtypes = [_P, C.c_int, _P, C.c_int64]
_lib.ot_state_cost.argtypes = [_P, C.POINTER(C.c_double), C.POINTER(C.c_double)]
_lib.ot_state_counters.argtypes = [_P, C.POINTER(C.c_int64), C.c_int32]
_lib.ot_shard_range.argtypes = [C.c_int64, C.c_int32, C.c_int32, C.POINTER(C.c_int64), C.POINTER(C.c_int64)]
_lib.ot_shard_create.argtypes = [_P, C.POINTER(OtProblem), C.POINTER(OtParams), C.c_int32, C.c_int32, C.POINTER(_P)]
_lib.ot_shard_slice.argtypes = [_P, C.c_int32, C.POINTER(C.c_int64), C.POINTER(C.c_int64)]
_lib.ot_shard_half_sweep.argtypes = [_P, C.c_int32, C.c_int32]
_lib.ot_shard_pack_bytes.argtypes = [_P, C.c_int32, C.c_int32, C.POINTER(C.c_size_t)]
_lib.ot_shard_pack_get.argtypes = [_P, C.c_int32, C.c_void_p]
_lib.ot_shard_pack_put.argtypes = [_P, C.c_int32, C.c_int32, C.c_void_p]
_lib.ot_shard_cert_partials.argtypes = [_P, C.POINTER(C.c_double)]
_lib.ot_set_tile_plan.argtypes = [C.c_int32, C.c_int32, C.c_int32, C.c_int32]
_lib.ot_get_tile_plan.argtypes = [C.c_int32, C.c_int32, C.POINTER(C.c_int32), C.POINTER(C.c_int32)]


class OtMarginalErrors(C.Structure):
    _fields_ = [(k, C.c_double) for k in ("row_l1", "row_max_abs", "row_max_rel", "col_l1", "col_max_abs",
                                          "col_max_rel", "eps")]


OT_PLAN_BEST, OT_PLAN_LATEST, OT_PLAN_INTERMEDIATE = range(3)
_lib.ot_plan_project.argtypes = [_P, C.c_int32, C.c_void_p, C.c_void_p, C.c_void_p, C.POINTER(OtMarginalErrors)]
_lib.ot_plan_round.argtypes = [_P, C.c_int32, C.POINTER(C.c_double), C.POINTER(C.c_double)]
_lib.ot_serve_create.argtypes = [_P, C.c_size_t, C.c_int32, C.c_uint64, C.POINTER(_P)]
_lib.ot_serve_submit.argtypes = [_P, C.POINTER(OtProblem), C.POINTER(OtParams), C.POINTER(C.c_uint64)]
_lib.ot_serve_poll.argtypes = [_P, C.c_uint64, _P, _P, C.POINTER(OtResult)]
_lib.ot_serve_wait.argtypes = [_P, C.c_uint64, C.c_double, _P, _P, C.POINTER(OtResult)]
_lib.ot_serve_cancel.argtypes = [_P, C.c_uint64]
_lib.ot_serve_stats.argtypes = [_P, C.POINTER(OtServeStats)]
_lib.ot_serve_reset_stats.argtypes = [_P]
_lib.ot_serve_destroy.argtypes = [_P]
_lib.ot_serve_profile_enable.argtypes = [_P, C.c_int]
_lib.ot_serve_profile_read.argtypes = [_P, C.c_int, C.POINTER(C.c_int64), C.POINTER(C.c_double),
                                       C.POINTER(C.c_double)]
_lib.ot_serve_profile_launches.argtypes = [_P, C.c_void_p, C.c_int64, C.POINTER(C.c_int64)]
_lib.ot_profile_enable.argtypes = [_P, C.c_int]
_lib.ot_profile_reset.argtypes = [_P]
_lib.ot_profile_read.argtypes = [_P, C.c_int, C.POINTER(C.c_int64), C.POINTER(C.c_double), C.POINTER(C.c_double)]
_lib.ot_launch_count.argtypes = [_P, C.POINTER(C.c_int64)]
_lib.ot_debug_set_wait_limit.argtypes = [_P, C.c_uint32]
_lib.ot_probe_pipes.argtypes = [C.c_int, C.c_int, C.POINTER(C.c_double), C.c_int]
_lib.ot_probe_exp2.argtypes = [C.c_int, C.c_int, C.c_void_p, C.c_void_p, C.c_int64]


class OTError(RuntimeError):
    def __init__(self, status: int, msg: str):
        super().__init__(f"{_lib.ot_status_str(status).decode()}: {msg}")
        self.status = status


def lib() -> C.CDLL:
    """The loaded ``libot.so`` (for callers that use the C ABI directly)."""
    return _lib


# --- argument marshalling -----------------------------------------------------------------
def _is_torch(t) -> bool:
    return type(t).__module__.startswith("torch")


def _host(arr, dtype) -> np.ndarray:
    return np.ascontiguousarray(np.asarray(arr, dtype=dtype))


def _ptr(arr) -> int:
    if _is_torch(arr):
        return int(arr.data_ptr())
    return int(arr.ctypes.data)


def make_problem(x, y, a, b, cost_scale: float = 0.0, omega: float = 0.0, zero_mass_floor: float = 0.0):
    """Build an ``ot_problem``.  Returns (struct, keepalive) — keep the second alive during calls."""
    dev = _is_torch(x)
    if dev:
        import torch
        x = x.to(torch.float32).contiguous()
        y = y.to(torch.float32).contiguous()
        a = a.to(torch.float64).contiguous()
        b = b.to(torch.float64).contiguous()
        n, d = (int(x.shape[0]), int(x.shape[1])) if x.dim() == 2 else (int(x.shape[0]), 1)
        m = int(y.shape[0])
    else:
        x = _host(x, np.float32)
        y = _host(y, np.float32)
        a = _host(a, np.float64)
        b = _host(b, np.float64)
        n, d = (x.shape[0], x.shape[1]) if x.ndim == 2 else (x.shape[0], 1)
        m = y.shape[0]
    p = OtProblem(n, m, d, 1 if dev else 0, _ptr(x), _ptr(y), _ptr(a), _ptr(b),
                  float(cost_scale), float(omega), float(zero_mass_floor))
    return p, (x, y, a, b)


def make_params(eps0=1.0, lam=1.0, max_iters=1000, cert_every=100, precision="mufu", tol_abs=0.0,
                tol_rel=0.0, time_budget_s=0.0, stream: int = 0, algorithm="bdrs", refine_on: float = 0.0,
                refine_tol: float = 0.0) -> OtParams:
    prm = OtParams()
    _lib.ot_params_default(C.byref(prm))
    prm.eps0 = float(eps0)
    prm.lam = float(lam)
    prm.max_iters = int(max_iters)
    prm.cert_every = int(cert_every)
    prm.precision = PRECISIONS[precision] if isinstance(precision, str) else int(precision)
    prm.tol_abs = float(tol_abs)
    prm.tol_rel = float(tol_rel)
    prm.time_budget_s = float(time_budget_s)
    prm.stream = int(stream)
    prm.algorithm = ALGORITHMS[algorithm] if isinstance(algorithm, str) else int(algorithm)
    prm.refine_on = float(refine_on)
    prm.refine_tol = float(refine_tol)
    return prm


class Context:
    """A solver context on one CUDA device (owns a stream)."""

    def __init__(self, device: int = 0):
        h = _P()
        st = _lib.ot_context_create(int(device), C.byref(h))
        if st != OT_OK:
            raise OTError(st, f"ot_context_create({device})")
        self._h = h

    @property
    def handle(self):
        return self._h

    def last_error(self) -> str:
        return _lib.ot_last_error(self._h).decode()

    def check(self, st: int, what: str):
        if st != OT_OK:
            raise OTError(st, f"{what}: {self.last_error()}")

    def close(self):
        if self._h:
            _lib.ot_context_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def solve(self, x, y, a, b, cost_scale=0.0, omega=0.0, zero_mass_floor=0.0, **params):
        """``ot_solve``: returns (f, g, result dict) — f, g numpy (host inputs) or torch (device inputs)."""
        prob, keep = make_problem(x, y, a, b, cost_scale, omega, zero_mass_floor)
        prm = make_params(**params)
        if prob.on_device:
            import torch
            f = torch.empty(prob.n, dtype=torch.float64, device=keep[0].device)
            g = torch.empty(prob.m, dtype=torch.float64, device=keep[0].device)
        else:
            f = np.empty(prob.n, np.float64)
            g = np.empty(prob.m, np.float64)
        res = OtResult()
        self.check(_lib.ot_solve(self._h, C.byref(prob), C.byref(prm), _ptr(f), _ptr(g), C.byref(res)),
                   "ot_solve")
        return f, g, res.as_dict()

    def state(self, x, y, a, b, cost_scale=0.0, omega=0.0, zero_mass_floor=0.0, **params) -> "State":
        return State(self, x, y, a, b, cost_scale, omega, zero_mass_floor, **params)


class State:
    """A resident solver state (``ot_state_*``, ``ot_step``, ``ot_certificate``)."""

    def __init__(self, ctx: Context, x, y, a, b, cost_scale=0.0, omega=0.0, zero_mass_floor=0.0, **params):
        self.ctx = ctx
        prob, keep = make_problem(x, y, a, b, cost_scale, omega, zero_mass_floor)
        prm = make_params(**params)
        h = _P()
        ctx.check(_lib.ot_state_create(ctx.handle, C.byref(prob), C.byref(prm), C.byref(h)), "ot_state_create")
        self._h = h
        self.n, self.m, self.d = int(prob.n), int(prob.m), int(prob.d)

    def close(self):
        if getattr(self, "_h", None):
            _lib.ot_state_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def step(self, n_iters: int) -> dict:
        res = OtResult()
        self.ctx.check(_lib.ot_step(self._h, int(n_iters), C.byref(res)), "ot_step")
        return res.as_dict()

    def certificate(self) -> dict:
        res = OtResult()
        self.ctx.check(_lib.ot_certificate(self._h, C.byref(res)), "ot_certificate")
        return res.as_dict()

    def get(self, which: int) -> np.ndarray:
        ln = self.n if which in (OT_LOG_ALPHA, OT_LOG_ALPHA_HAT, OT_F_CERT, OT_F_BEST) else self.m
        out = np.empty(ln, np.float64)
        k = C.c_int64()
        self.ctx.check(_lib.ot_state_get(self._h, int(which), out.ctypes.data, C.byref(k)), "ot_state_get")
        return out

    @property
    def k(self) -> int:
        k = C.c_int64()
        self.ctx.check(_lib.ot_state_get(self._h, OT_LOG_ALPHA, None, C.byref(k)), "ot_state_get")
        return int(k.value)

    def set(self, which: int, values, k: int):
        v = _host(values, np.float64)
        self.ctx.check(_lib.ot_state_set(self._h, int(which), v.ctypes.data, int(k)), "ot_state_set")

    def project(self, plan: int = OT_PLAN_BEST):
        """``ot_plan_project``: (y_hat [n, d] float32, row sums [n], column sums [m], errors dict)."""
        y_hat = np.empty((self.n, self.d), np.float32)
        row = np.empty(self.n, np.float64)
        col = np.empty(self.m, np.float64)
        err = OtMarginalErrors()
        self.ctx.check(_lib.ot_plan_project(self._h, int(plan), y_hat.ctypes.data, row.ctypes.data, col.ctypes.data,
                                            C.byref(err)), "ot_plan_project")
        return y_hat, row, col, {k: getattr(err, k) for k, _ in OtMarginalErrors._fields_}

    def round_cost(self, plan: int = OT_PLAN_BEST):
        """``ot_plan_round``: (cost of the rounded feasible plan, cost of the unrounded plan)."""
        cr, cu = C.c_double(), C.c_double()
        self.ctx.check(_lib.ot_plan_round(self._h, int(plan), C.byref(cr), C.byref(cu)), "ot_plan_round")
        return cr.value, cu.value

    def counters(self) -> dict:
        """``ot_state_counters``: shift-hint misses, fast-sweep tile recomputes, micro-split counts."""
        out = (C.c_int64 * 10)()
        self.ctx.check(_lib.ot_state_counters(self._h, out, 10), "ot_state_counters")
        v = list(out)
        return {"hint_miss_rows": v[0:2], "hint_miss_cols": v[2:4], "tile_recomputes": v[4],
                "splits_fast": (v[5], v[6]), "splits_cert": (v[7], v[8]), "tiles_refined": v[9]}

    def cost(self):
        kap, om = C.c_double(), C.c_double()
        self.ctx.check(_lib.ot_state_cost(self._h, C.byref(kap), C.byref(om)), "ot_state_cost")
        return kap.value, om.value


def shard_range(np_: int, rank: int, world: int):
    """``ot_shard_range``: the points [p0, p1) of a side of np_ points that rank of world updates."""
    p0, p1 = C.c_int64(), C.c_int64()
    st = _lib.ot_shard_range(int(np_), int(rank), int(world), C.byref(p0), C.byref(p1))
    if st != OT_OK:
        raise OTError(st, "ot_shard_range")
    return int(p0.value), int(p1.value)


class ShardState(State):
    """One slice of a row-sharded solve (``ot_shard_*``); see ``paper_2609_33814_b300.shard``."""

    def __init__(self, ctx: Context, x, y, a, b, rank: int, world: int, cost_scale=0.0, omega=0.0,
                 zero_mass_floor=0.0, **params):
        self.ctx = ctx
        prob, keep = make_problem(x, y, a, b, cost_scale, omega, zero_mass_floor)
        prm = make_params(**params)
        h = _P()
        ctx.check(_lib.ot_shard_create(ctx.handle, C.byref(prob), C.byref(prm), int(rank), int(world), C.byref(h)),
                  "ot_shard_create")
        self._h = h
        self.n, self.m, self.d = int(prob.n), int(prob.m), int(prob.d)
        self.rank, self.world = int(rank), int(world)

    def slice(self, side: int):
        p0, p1 = C.c_int64(), C.c_int64()
        self.ctx.check(_lib.ot_shard_slice(self._h, int(side), C.byref(p0), C.byref(p1)), "ot_shard_slice")
        return int(p0.value), int(p1.value)

    def half_sweep(self, side: int, cert: bool):
        self.ctx.check(_lib.ot_shard_half_sweep(self._h, int(side), 1 if cert else 0), "ot_shard_half_sweep")

    def pack_bytes(self, side: int, rank: int) -> int:
        nb = C.c_size_t()
        self.ctx.check(_lib.ot_shard_pack_bytes(self._h, int(side), int(rank), C.byref(nb)), "ot_shard_pack_bytes")
        return int(nb.value)

    def pack_get(self, side: int) -> np.ndarray:
        buf = np.empty(self.pack_bytes(side, self.rank), np.uint8)
        self.ctx.check(_lib.ot_shard_pack_get(self._h, int(side), buf.ctypes.data), "ot_shard_pack_get")
        return buf

    def pack_put(self, side: int, rank: int, buf: np.ndarray):
        b = np.ascontiguousarray(buf, np.uint8)
        assert b.size == self.pack_bytes(side, rank)
        self.ctx.check(_lib.ot_shard_pack_put(self._h, int(side), int(rank), b.ctypes.data), "ot_shard_pack_put")

    def cert_partials(self) -> np.ndarray:
        out = (C.c_double * 5)()
        self.ctx.check(_lib.ot_shard_cert_partials(self._h, out), "ot_shard_cert_partials")
        return np.array(list(out))


class Server:
    """Continuous-batching server (``ot_serve_*``); thread-safe.  Results come back on the host."""

    def __init__(self, ctx: Context, hbm_budget_bytes: int = 8 << 30, max_slots: int = 64, stream: int = 0):
        self.ctx = ctx
        h = _P()
        st = _lib.ot_serve_create(ctx.handle, int(hbm_budget_bytes), int(max_slots), int(stream), C.byref(h))
        if st != OT_OK:
            raise OTError(st, "ot_serve_create")
        self._h = h
        self._sizes = {}

    def submit(self, x, y, a, b, cost_scale=0.0, omega=0.0, zero_mass_floor=0.0, **params) -> int:
        prob, keep = make_problem(x, y, a, b, cost_scale, omega, zero_mass_floor)
        prm = make_params(**params)
        rid = C.c_uint64()
        st = _lib.ot_serve_submit(self._h, C.byref(prob), C.byref(prm), C.byref(rid))
        if st != OT_OK:
            raise OTError(st, "ot_serve_submit")
        self._sizes[rid.value] = (int(prob.n), int(prob.m))
        return int(rid.value)

    def _collect(self, fn, rid, *extra):
        n, m = self._sizes[rid]
        f = np.empty(n, np.float64)
        g = np.empty(m, np.float64)
        res = OtResult()
        st = fn(self._h, C.c_uint64(rid), *extra, f.ctypes.data, g.ctypes.data, C.byref(res))
        if st == OT_EBUSY:
            return None
        self._sizes.pop(rid, None)
        if st != OT_OK:
            raise OTError(st, f"request {rid}")
        return f, g, res.as_dict()

    def poll(self, rid: int):
        """(f, g, result) when finished, None while queued or running."""
        return self._collect(_lib.ot_serve_poll, rid)

    def wait(self, rid: int, timeout_s: float = -1.0):
        return self._collect(_lib.ot_serve_wait, rid, C.c_double(timeout_s))

    def cancel(self, rid: int):
        st = _lib.ot_serve_cancel(self._h, C.c_uint64(rid))
        if st != OT_OK:
            raise OTError(st, f"cancel {rid}")

    def stats(self) -> dict:
        s = OtServeStats()
        _lib.ot_serve_stats(self._h, C.byref(s))
        return s.as_dict()

    def reset_stats(self):
        _lib.ot_serve_reset_stats(self._h)

    def profile(self, on: bool):
        _lib.ot_serve_profile_enable(self._h, 1 if on else 0)

    def kernel_stats(self, kind: int):
        """(launches, entries, ms) since the last reset of kind 0 (fast iterations) or 1 (certificate
        iterations); entries count both sweeps of every iteration."""
        n, e, ms = C.c_int64(), C.c_double(), C.c_double()
        _lib.ot_serve_profile_read(self._h, int(kind), C.byref(n), C.byref(e), C.byref(ms))
        return n.value, e.value, ms.value

    def launch_log(self) -> np.ndarray:
        """Per fast launch since the last reset: rows (implicit entries, ms, instances in the lane)."""
        n = C.c_int64()
        _lib.ot_serve_profile_launches(self._h, None, 0, C.byref(n))
        out = np.zeros((n.value, 3), np.float64)
        if n.value:
            _lib.ot_serve_profile_launches(self._h, out.ctypes.data, n.value, C.byref(n))
        return out

    def close(self):
        if getattr(self, "_h", None):
            _lib.ot_serve_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def probe_exp2(x, method: str = "poly", device: int = 0) -> np.ndarray:
    """exp2 of the float32 array x by the sweep's SFU ("mufu") or FMA-pipe polynomial ("poly")."""
    xs = np.ascontiguousarray(x, np.float32)
    out = np.empty_like(xs)
    st = _lib.ot_probe_exp2(int(device), {"mufu": 0, "poly": 1}[method], xs.ctypes.data, out.ctypes.data,
                            int(xs.size))
    if st != OT_OK:
        raise OTError(st, "ot_probe_exp2")
    return out




def set_tile_plan(d: int, precision: str, R: int, ch: int) -> None:
    """``ot_set_tile_plan``: the (R, CH) of the sweep kernels of (d, precision); R = 0 resets."""
    st = _lib.ot_set_tile_plan(int(d), PRECISIONS[precision], int(R), int(ch))
    if st != OT_OK:
        raise OTError(st, f"ot_set_tile_plan({d}, {precision}, {R}, {ch})")


def get_tile_plan(d: int, precision: str):
    """``ot_get_tile_plan``: the (R, CH) instances of (d, precision) use now."""
    R, ch = C.c_int32(), C.c_int32()
    st = _lib.ot_get_tile_plan(int(d), PRECISIONS[precision], C.byref(R), C.byref(ch))
    if st != OT_OK:
        raise OTError(st, "ot_get_tile_plan")
    return int(R.value), int(ch.value)
