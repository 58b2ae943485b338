"""Seeded synthetic velocity distributions for the collision-operator workloads.

This module holds input distributions only: closed-form densities f(v) and the
seeded draws of their parameters.  It contains none of the spectral method's
arithmetic (no maps, no Chebyshev functions, no quadrature, no collision
operator).  Both the CUDA path and the CPU oracle take their inputs from here;
each projects f onto its own trial space.

Workloads (sizes in the paper's notation: N = highest mode per axis, M sphere points):

* ``c1_2d_maxwell``:  2D, Maxwell molecules (gamma = 0), N = 16, S = 2, M = 8.
  f = sum of two isotropic Maxwellians of mass 1/2 (as in the two-Maxwellian
  moment test of Section 5.1.2); centres uniform in [-1.5, 1.5]^2,
  temperatures uniform in [0.5, 1.5].
* ``c2_2d_vhs``:  2D, hard spheres (gamma = 1), N = 64, S = 3, M = 32.
  Three Maxwellians of mass 1/3 plus a positive Gaussian-windowed perturbation
  of amplitude 0.1:  0.1 u(v) exp(-|v|^2/2)/(2 pi), with
  u = (1/8) sum_n (1 + cos(kappa_n . v + phi_n))/2 in [0, 1].
* ``c3_3d_bkw``:  3D, Maxwell molecules, N = 16, S = 2, M = 32: the 3D BKW
  solution of Section 5.2 at K = 3/5 (its earliest non-negative profile).
* ``c4_3d_bimaxwell``:  3D, gamma = 0.5, N = 24, S = 3, M = 32: an anisotropic
  bi-Maxwellian with temperatures (0.6, 1.4, 1.4) and a seeded shift in
  [-0.5, 0.5]^3.
* ``c5_batched_2d``:  4096 independent 2D cells, N in {16, 24, 32}, M in
  {8, 16, 32}, gamma in {0, 1}, S = 3, f = 1-3 Maxwellians of equal mass.

Seeds: numpy ``default_rng(2105 + index)`` with the index of the workload in
the list above (0-based).
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field

import numpy as np


def maxwellian(pts, rho, centre, temp):
    """rho (2 pi T)^(-d/2) exp(-|v - V|^2 / (2T)) at pts (P, d)."""
    pts = np.asarray(pts, dtype=np.float64)
    d = pts.shape[1]
    diff = pts - np.asarray(centre, dtype=np.float64)[None, :]
    return rho * (2 * math.pi * temp) ** (-d / 2) * np.exp(-np.sum(diff * diff, axis=1) / (2 * temp))


def bkw_2d(pts, t=None, K=None):
    """2D BKW profile of Section 5.1.1 (B = 1/(2 pi)), K = 1 - exp(-t/8)/2 unless K is given."""
    if K is None:
        K = 1 - math.exp(-t / 8) / 2
    pts = np.asarray(pts, dtype=np.float64)
    v2 = np.sum(pts * pts, axis=1)
    return (1 / (2 * math.pi * K * K)) * np.exp(-v2 / (2 * K)) * (2 * K - 1 + (1 - K) / (2 * K) * v2)


def bkw_3d(pts, t=None, K=None):
    """3D BKW profile of Section 5.2 (B = 1/(4 pi)), K = 1 - exp(-t/6) unless K is given."""
    if K is None:
        K = 1 - math.exp(-t / 6)
    pts = np.asarray(pts, dtype=np.float64)
    v2 = np.sum(pts * pts, axis=1)
    return (1 / (2 * (2 * math.pi * K) ** 1.5)) * np.exp(-v2 / (2 * K)) * ((5 * K - 3) / K + (1 - K) / (K * K) * v2)


@dataclass
class Workload:
    name: str
    d: int
    N: int
    M: int
    S: float
    gamma: float
    density: object = field(repr=False)  # callable pts (P, d) -> f (P,)
    note: str = ""

    def __call__(self, pts):
        return self.density(pts)


def _mixture(rng, d, count, lo=-1.5, hi=1.5, tlo=0.5, thi=1.5):
    comps = []
    for _ in range(count):
        centre = rng.uniform(lo, hi, size=d)
        temp = rng.uniform(tlo, thi)
        comps.append((1.0 / count, centre, temp))
    return comps


def _mix_density(comps):
    def f(pts):
        out = np.zeros(np.asarray(pts).shape[0])
        for rho, c, t in comps:
            out += maxwellian(pts, rho, c, t)
        return out
    return f


def c1_2d_maxwell() -> Workload:
    rng = np.random.default_rng(2105 + 0)
    comps = _mixture(rng, 2, 2)
    return Workload("c1_2d_maxwell_N16_M8", 2, 16, 8, 2.0, 0.0, _mix_density(comps),
                    "two Maxwellians, mass 1/2 each")


def c2_2d_vhs() -> Workload:
    rng = np.random.default_rng(2105 + 1)
    comps = _mixture(rng, 2, 3)
    kappa = rng.normal(size=(8, 2))
    phase = rng.uniform(0, 2 * math.pi, size=8)
    base = _mix_density(comps)

    def f(pts):
        pts = np.asarray(pts, dtype=np.float64)
        u = np.mean((1 + np.cos(pts @ kappa.T + phase[None, :])) / 2, axis=1)
        window = np.exp(-np.sum(pts * pts, axis=1) / 2) / (2 * math.pi)
        return base(pts) + 0.1 * u * window
    return Workload("c2_2d_vhs_N64_M32", 2, 64, 32, 3.0, 1.0, f,
                    "three Maxwellians + 0.1 Gaussian-windowed positive perturbation")


def c3_3d_bkw(K: float = 0.6) -> Workload:
    return Workload("c3_3d_bkw_N16_M32", 3, 16, 32, 2.0, 0.0, lambda p: bkw_3d(p, K=K),
                    f"3D BKW profile at K={K}")


def c4_3d_bimaxwell() -> Workload:
    rng = np.random.default_rng(2105 + 3)
    shift = rng.uniform(-0.5, 0.5, size=3)
    temps = np.array([0.6, 1.4, 1.4])

    def f(pts):
        pts = np.asarray(pts, dtype=np.float64)
        q = np.sum((pts - shift[None, :]) ** 2 / temps[None, :], axis=1)
        return (2 * math.pi) ** -1.5 / math.sqrt(np.prod(temps)) * np.exp(-q / 2)
    return Workload("c4_3d_bimaxwell_N24_M32", 3, 24, 32, 3.0, 0.5, f,
                    "bi-Maxwellian T=(0.6,1.4,1.4), seeded shift")


def c5_batched_2d(ncell: int = 4096):
    """Per-cell (N, M, gamma, density) lists for the batched 2D workload."""
    rng = np.random.default_rng(2105 + 4)
    Ns = rng.choice([16, 24, 32], size=ncell)
    Ms = rng.choice([8, 16, 32], size=ncell)
    gam = np.where(rng.uniform(size=ncell) < 0.5, 0.0, 1.0)
    cells = []
    for c in range(ncell):
        count = int(rng.integers(1, 4))
        comps = _mixture(rng, 2, count)
        cells.append(Workload(f"cell{c}", 2, int(Ns[c]), int(Ms[c]), 3.0, float(gam[c]),
                              _mix_density(comps), f"{count} Maxwellians"))
    return cells


ALL = {
    "c1": c1_2d_maxwell,
    "c2": c2_2d_vhs,
    "c3": c3_3d_bkw,
    "c4": c4_3d_bimaxwell,
}
