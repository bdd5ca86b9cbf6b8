"""Float64 reference of the differentiable short-range trajectory.

TEST INFRASTRUCTURE (see the package docstring).

Trajectory: ``steps`` repetitions of the short-range kick followed by a drift
(the kick and stream maps of the paper's split-operator step, Eq. 6):

    v_{k+1} = v_k + dt a(x_k, m),   x_{k+1} = x_k + dt v_{k+1},

with positions kept unwrapped (the force uses the minimum image, so it is
periodic in x).  Loss: sum_i w_i . (x_S,i - x_0,i)^2 (componentwise square),
w seeded.  The gradient is taken by hand in reverse order with the oracle's
float64 force adjoint; ``finite_difference`` gives central differences of the
same float64 loss.
"""

from __future__ import annotations

import numpy as np

from . import kick_drift, sr_force, sr_force_adjoint


def _force(x, m, L, eps, rcut, c):
    return sr_force(x[:, 0], x[:, 1], x[:, 2], m, L, eps, rcut, c)


def trajectory(x0, v0, m, L, eps, rcut, c, dt, steps):
    xs = [np.array(x0, dtype=np.float64)]
    v = np.array(v0, dtype=np.float64)
    for _ in range(steps):
        a = _force(xs[-1], m, L, eps, rcut, c)
        v, xn = kick_drift(v, a, dt, xs[-1], dt)
        xs.append(xn)
    return xs, v


def loss(x0, v0, m, L, eps, rcut, c, dt, steps, w) -> float:
    xs, _ = trajectory(x0, v0, m, L, eps, rcut, c, dt, steps)
    dx = xs[-1] - xs[0]
    return float(np.sum(np.asarray(w, np.float64) * dx * dx))


def gradient(x0, v0, m, L, eps, rcut, c, dt, steps, w):
    """(dL/dx0 [N,3], dL/dv0 [N,3], dL/dm [N]) in float64, by reverse accumulation."""
    w = np.asarray(w, np.float64)
    m = np.asarray(m, np.float64)
    xs, _ = trajectory(x0, v0, m, L, eps, rcut, c, dt, steps)
    g_last = 2.0 * w * (xs[-1] - xs[0])
    gx = g_last.copy()            # cotangent of x_{k+1}, starting at k+1 = S
    gx0_direct = -g_last          # x_0 also enters the loss directly
    gv = np.zeros_like(gx)        # cotangent of v_{k+1}
    gm = np.zeros(m.shape[0])
    for k in range(steps - 1, -1, -1):
        # x_{k+1} = x_k + dt v_{k+1}
        gv = gv + dt * gx
        # v_{k+1} = v_k + dt a(x_k): cotangent of a_k is dt gv
        lam = dt * gv
        xk = xs[k]
        g_ax, g_am = sr_force_adjoint(xk[:, 0], xk[:, 1], xk[:, 2], m, L, eps, rcut, c, lam)
        gx = gx + g_ax            # cotangent of x_k
        gm = gm + g_am
        # gv passes through unchanged to v_k
    return gx + gx0_direct, gv, gm


def finite_difference(x0, v0, m, L, eps, rcut, c, dt, steps, w, which, index, h):
    """Central difference of the loss along one coordinate.

    which: 'x' or 'v' (index = (particle, axis)) or 'm' (index = particle).
    """
    x0 = np.array(x0, np.float64)
    v0 = np.array(v0, np.float64)
    m = np.array(m, np.float64)
    vals = []
    for sgn in (1.0, -1.0):
        xp, vp, mp = x0.copy(), v0.copy(), m.copy()
        if which == "x":
            xp[index] += sgn * h
        elif which == "v":
            vp[index] += sgn * h
        else:
            mp[index] += sgn * h
        vals.append(loss(xp, vp, mp, L, eps, rcut, c, dt, steps, w))
    return (vals[0] - vals[1]) / (2.0 * h)
