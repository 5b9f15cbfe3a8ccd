"""Seeded synthetic input generators shared by the CUDA path's tests/bench and the oracle.

This module holds none of the method's arithmetic: it only draws random numbers
(NumPy PCG64 streams keyed by a seed) and shapes them into arrays.  Everything
that depends on the paper's method (grids, metrics, operators, truncation) lives
either in the CUDA library or in the oracle, never here.
"""
from __future__ import annotations

import numpy as np


def rng(seed: int) -> np.random.Generator:
    return np.random.Generator(np.random.PCG64(int(seed)))


def bond_profile(n: int, chi: int, d: int = 2) -> list[int]:
    """Bond sizes r_0..r_n = min(d^k, d^(n-k), chi) (the profile of eq:simpleMPS)."""
    out = []
    for k in range(n + 1):
        out.append(int(min(d ** min(k, 60), d ** min(n - k, 60), chi)))
    return out


def random_cores(n: int, chi: int, seed: int, d: int = 2, bonds: list[int] | None = None,
                 scale: float = 1.0) -> list[np.ndarray]:
    """i.i.d. N(0, scale^2) cores of shape (r_{k-1}, d, r_k), row-major, float64."""
    g = rng(seed)
    b = bonds if bonds is not None else bond_profile(n, chi, d)
    return [scale * g.standard_normal((b[k], d, b[k + 1])) for k in range(n)]


def random_mpo_cores(n: int, w: int, seed: int, d: int = 2) -> list[np.ndarray]:
    g = rng(seed)
    b = [1] + [w] * (n - 1) + [1]
    return [g.standard_normal((b[k], d, d, b[k + 1])) for k in range(n)]


def gaussian_field(n_eta: int, n_xi: int, seed: int, amp: float) -> np.ndarray:
    """i.i.d. N(0, amp^2) values on the (2^n_eta, 2^n_xi) interior grid, row = eta index i."""
    g = rng(seed)
    return amp * g.standard_normal((2 ** n_eta, 2 ** n_xi))


def dense_vector(n: int, seed: int) -> np.ndarray:
    return rng(seed).standard_normal(2 ** n)


def wake_field(n_eta: int, n_xi: int, seed: int) -> tuple[np.ndarray, np.ndarray]:
    """A smooth synthetic (u, v) pair on the (2^n_eta, 2^n_xi) index grid, shaped like a developed
    cylinder wake in the unit-square coordinates eta = (i + 1/2) / N_eta (radial) and
    xi = j / N_xi (angular, periodic; xi = 0 downstream): u = 1 outside, a thin layer where u
    drops to 0 at eta = 0, a velocity deficit around xi = 0 widening outwards, and six seeded
    travelling-wave packets in u and v (amplitude ~5e-2).  Every term is smooth and periodic in
    xi, so the field's tensor-train spectrum decays steadily (no flat tail at a bond cap)."""
    g = rng(seed)
    eta = (np.arange(2 ** n_eta) + 0.5) / 2 ** n_eta
    xi = np.arange(2 ** n_xi) / 2 ** n_xi
    E, X = np.meshgrid(eta, xi, indexing="ij")
    wake = np.exp(-(np.sin(np.pi * X) / (0.12 + 0.2 * E)) ** 2)
    u = 1.0 - np.exp(-E / 0.02) - 0.3 * wake * (1.0 - np.exp(-E / 0.1))
    v = np.zeros_like(u)
    for f in (u, v):
        for _ in range(6):
            a = 0.05 * g.standard_normal()
            e0 = g.uniform(0.15, 0.85)
            m = int(g.integers(1, 5))
            ph = g.uniform(0.0, 1.0)
            f += a * np.exp(-((E - e0) / 0.05) ** 2) * np.cos(2.0 * np.pi * m * (X - ph))
    return u, v
