"""Seeded synthetic workloads for the optimal-transport solver and its tests.

This module only *draws inputs*: point clouds, histograms and request streams.
It holds none of the solver's arithmetic (no cost matrix, no log-sum-exp, no
scaling update), so both the FP64 oracle tests and the CUDA product path can
use it without sharing any of the method's code.

Workload shapes follow the paper's experiments:

* grid histograms on an ``s x s`` pixel grid with integer pixel coordinates
  ``z_i in {0..s-1}^2`` and the paper's normalised squared-Euclidean cost
  ``C_ij = ||z_i - z_j||^2 / (2 (s-1)^2)`` (Appendix G, "Data and ground
  cost"); the normalisation is returned as ``kappa`` so that
  ``C_ij = kappa * ||z_i - z_j||^2``;
* histogram classes standing in for the DOTmark classes (which are not
  available here): uniform-random, 1-5 component Gaussian mixtures,
  heavy-tailed Cauchy-like densities and 90%-sparse histograms whose zeros are
  floored at 1e-15 the way the paper treats zero-mass pixels (Appendix G);
* RGB colour clouds standing in for the colour-transfer photographs
  (Appendix G, "Pixel-level OT formulation"): colours in [0,1]^3 drawn from
  an 8-component Gaussian mixture, clipped to the cube, uniform weights.

Every generator takes an explicit integer seed and returns float32
coordinates (the solver's input precision) and float64 weights.
"""
from __future__ import annotations

import dataclasses
from typing import List, Optional

import numpy as np

HIST_CLASSES = ("uniform", "gaussmix", "cauchy", "sparse")
ZERO_MASS_FLOOR = 1e-15


def _rng(seed: int) -> np.random.Generator:
    return np.random.Generator(np.random.PCG64(int(seed)))


def grid_points(s: int) -> np.ndarray:
    """Integer pixel coordinates of an ``s x s`` grid, row-major, float32 (n=s*s, 2)."""
    iy, ix = np.meshgrid(np.arange(s), np.arange(s), indexing="ij")
    return np.stack([ix.ravel(), iy.ravel()], axis=1).astype(np.float32)


def grid_kappa(s: int) -> float:
    """Cost scale so that kappa*||z_i-z_j||^2 equals the paper's grid cost in [0,1]."""
    return 1.0 / (2.0 * (s - 1) ** 2) if s > 1 else 1.0


def uniform_weights(n: int, seed: int) -> np.ndarray:
    """Weights drawn as U[0,1) + 1e-6, normalised to sum 1 (float64)."""
    w = _rng(seed).random(n) + 1e-6
    return w / w.sum()


def histogram(s: int, cls: str, seed: int) -> np.ndarray:
    """A seeded ``s x s`` histogram of class ``cls``, flattened row-major, sum 1, float64."""
    rng = _rng(seed)
    n = s * s
    iy, ix = np.meshgrid(np.arange(s), np.arange(s), indexing="ij")
    u = np.stack([ix.ravel(), iy.ravel()], axis=1).astype(np.float64) / max(s - 1, 1)
    if cls == "uniform":
        w = rng.random(n) + 1e-6
    elif cls == "gaussmix":
        k = int(rng.integers(1, 6))
        centres = rng.random((k, 2))
        sig = rng.uniform(0.03, 0.25, size=k)
        mix = rng.dirichlet(np.ones(k))
        w = np.zeros(n)
        for c, sg, p in zip(centres, sig, mix):
            d2 = ((u - c) ** 2).sum(1)
            w += p * np.exp(-0.5 * d2 / sg ** 2) / (2 * np.pi * sg ** 2)
        w += 1e-12
    elif cls == "cauchy":
        k = int(rng.integers(1, 4))
        centres = rng.random((k, 2))
        gam = rng.uniform(0.02, 0.2, size=k)
        w = np.zeros(n)
        for c, g in zip(centres, gam):
            d2 = ((u - c) ** 2).sum(1)
            w += (1.0 + d2 / g ** 2) ** -1.5
    elif cls == "sparse":
        w = rng.random(n) + 1e-6
        mask = rng.random(n) < 0.9
        w[mask] = 0.0
        if w.sum() == 0.0:
            w[int(rng.integers(0, n))] = 1.0
        w = w / w.sum()
        w = np.maximum(w, ZERO_MASS_FLOOR)
    else:
        raise ValueError(f"unknown histogram class {cls!r}")
    return w / w.sum()


def rgb_cloud(n: int, seed: int, components: int = 8) -> np.ndarray:
    """``n`` colours in [0,1]^3 from a seeded Gaussian mixture, clipped, float32 (n, 3)."""
    rng = _rng(seed)
    means = rng.random((components, 3))
    sig = rng.uniform(0.03, 0.2, size=(components, 3))
    mix = rng.dirichlet(np.ones(components))
    lab = rng.choice(components, size=n, p=mix)
    pts = means[lab] + sig[lab] * rng.standard_normal((n, 3))
    return np.clip(pts, 0.0, 1.0).astype(np.float32)


def random_cloud(n: int, d: int, seed: int, lo: float = 0.0, hi: float = 1.0) -> np.ndarray:
    """``n`` points uniform in [lo,hi]^d, float32."""
    return _rng(seed).uniform(lo, hi, size=(n, d)).astype(np.float32)


@dataclasses.dataclass
class Problem:
    """One OT instance: sources x (n,d) with weights a, targets y (m,d) with weights b.

    ``kappa`` scales the squared-Euclidean cost (C = kappa*||x-y||^2) and
    ``omega`` is an upper bound on the cost oscillation (max C - min C).
    """
    x: np.ndarray
    y: np.ndarray
    a: np.ndarray
    b: np.ndarray
    kappa: float
    omega: float
    name: str = ""

    @property
    def n(self) -> int:
        return int(self.x.shape[0])

    @property
    def m(self) -> int:
        return int(self.y.shape[0])

    @property
    def d(self) -> int:
        return int(self.x.shape[1])


def grid_problem(s: int, seed: int, cls_a: str = "uniform", cls_b: Optional[str] = None) -> Problem:
    """A pair of ``s x s`` histograms (seeds ``seed`` and ``seed+1``) with the paper's grid cost.

    With the normalisation kappa = 1/(2(s-1)^2) the cost lies in [0,1], so
    omega = 1 bounds its oscillation.
    """
    z = grid_points(s)
    if cls_b is None:
        cls_b = cls_a
    if cls_a == "uniform" and cls_b == "uniform":
        a = uniform_weights(s * s, seed)
        b = uniform_weights(s * s, seed + 1)
    else:
        a = histogram(s, cls_a, seed)
        b = histogram(s, cls_b, seed + 1)
    return Problem(z, z.copy(), a, b, grid_kappa(s), 1.0, f"grid{s}_{cls_a}_{cls_b}_{seed}")


def rgb_problem(n: int, seed: int, m: Optional[int] = None) -> Problem:
    """Colour-transfer stand-in: two seeded RGB mixtures, uniform weights.

    ``kappa`` is left at 1/3 (the cube's squared diameter, an upper bound on
    every pair cost) so that C lies in [0,1] and omega = 1; callers that want
    the paper's exact max-cost normalisation compute it and replace kappa.
    """
    m = n if m is None else m
    x = rgb_cloud(n, seed)
    y = rgb_cloud(m, seed + 1)
    a = np.full(n, 1.0 / n)
    b = np.full(m, 1.0 / m)
    return Problem(x, y, a, b, 1.0 / 3.0, 1.0, f"rgb{n}x{m}_{seed}")


@dataclasses.dataclass
class Request:
    """One request of a serving stream: arrival time (s) and its problem recipe."""
    arrival_s: float
    s: int
    cls_a: str
    cls_b: str
    seed: int


def serving_stream(count: int, seed: int, rate_per_s: float,
                   sizes=(32, 64, 128), size_p=(0.50, 0.35, 0.15)) -> List[Request]:
    """``count`` requests with Poisson arrivals at ``rate_per_s``; grid sizes and
    histogram classes drawn per request (the mixed-size serving workload)."""
    rng = _rng(seed)
    gaps = rng.exponential(1.0 / rate_per_s, size=count)
    t = np.cumsum(gaps) - gaps[0]
    out = []
    for i in range(count):
        s = int(rng.choice(np.asarray(sizes), p=np.asarray(size_p)))
        ca = HIST_CLASSES[int(rng.integers(0, len(HIST_CLASSES)))]
        cb = HIST_CLASSES[int(rng.integers(0, len(HIST_CLASSES)))]
        out.append(Request(float(t[i]), s, ca, cb, int(rng.integers(0, 2 ** 31 - 2))))
    return out


def request_problem(req: Request) -> Problem:
    return grid_problem(req.s, req.seed, req.cls_a, req.cls_b)
