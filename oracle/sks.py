"""Float64 reference of the short-range sub-cycles of the split-operator step.

TEST INFRASTRUCTURE (see the package docstring).

One sub-cycle is the symmetric stream-kick-stream map of the paper's Eq. 6
for the short-range force alone: x += h/2 v (wrapped into [0, L)), a = a(x),
v += h a, x += h/2 v (wrapped).  Energy = sum m v^2 / 2 + sum m phi / 2.
"""

from __future__ import annotations

import numpy as np

from . import sr_force, sr_potential


def energy(x, v, m, L, eps, rcut, c) -> tuple[float, float]:
    phi = sr_potential(x[:, 0], x[:, 1], x[:, 2], m, L, eps, rcut, c)
    return float(0.5 * np.sum(m[:, None] * v * v)), float(0.5 * np.sum(m * phi))


def subcycles(x, v, m, L, eps, rcut, c, h, n_c):
    """(x, v, [(kinetic, potential) after each sub-cycle]) in float64."""
    x = np.array(x, np.float64)
    v = np.array(v, np.float64)
    m = np.asarray(m, np.float64)
    hist = []
    for _ in range(n_c):
        x = np.mod(x + 0.5 * h * v, L)
        a = sr_force(x[:, 0], x[:, 1], x[:, 2], m, L, eps, rcut, c)
        v = v + h * a
        x = np.mod(x + 0.5 * h * v, L)
        hist.append(energy(x, v, m, L, eps, rcut, c))
    return x, v, hist
