"""Default coefficients of the grid-force polynomial f_grid(s) = poly[5](s).

The paper (Sec. II, force-split discussion, and Eq. 7) obtains the filtered
grid force numerically, fits it with the right small- and large-distance
asymptotics, and replaces the fit by a fifth-order polynomial in s = r.r over
the short-range region.  It prints neither the fit nor the coefficients.  The
force law takes the six coefficients as an input, so any set is valid for the
short-range path; this module supplies a physically motivated default:

* The grid force is modelled as the force of a Gaussian-smoothed unit point
  mass, g(s) d with g(s) = [erf(r/se) - 2 r/(se sqrt(pi)) exp(-s/se^2)] / r^3.
  It is finite at r = 0 (value 4/(3 sqrt(pi) se^3)) and tends to r^-3 at
  large r, the asymptotics the paper asks of its fit.
* se^2 = sigma^2 + (n_s + 4) Delta^2 / 6 matches the second moment of the
  paper's spectral filter exp(-k^2 sigma^2/4) sinc^n_s(k Delta/2) (Eq. 5,
  with sigma = 0.8, n_s = 3) times the CIC deposit and interpolation windows
  (two sinc^2 factors per axis), Delta = 1 grid unit.
* poly is the float64 least-squares fit of degree 5 in s to g on Chebyshev
  nodes of [0, r_c^2], with the one equality constraint
  poly(r_c^2) = (r_c^2 + eps)^-3/2, so that f_SR = (s + eps)^-3/2 - poly(s)
  vanishes at the cutoff and the force is continuous there.
"""

from __future__ import annotations

import math

import numpy as np

SIGMA = 0.8
N_S = 3
DELTA = 1.0


def sigma_eff(sigma: float = SIGMA, n_s: int = N_S, delta: float = DELTA) -> float:
    return math.sqrt(sigma * sigma + (n_s + 4) * delta * delta / 6.0)


def gaussian_grid_force(s: np.ndarray, se: float | None = None) -> np.ndarray:
    """g(s) of a Gaussian-smoothed unit point mass (force = g(s) d), float64."""
    if se is None:
        se = sigma_eff()
    s = np.asarray(s, dtype=np.float64)
    r = np.sqrt(s)
    out = np.empty_like(r)
    small = r < 1e-3 * se
    # series of erf near 0: g = 4/(3 sqrt(pi) se^3) * (1 - 3/5 x^2 + ...), x = r/se
    x2 = s[small] / (se * se)
    out[small] = 4.0 / (3.0 * math.sqrt(math.pi) * se ** 3) * (1.0 - 0.6 * x2)
    rl = r[~small]
    erf = np.array([math.erf(v / se) for v in rl])
    out[~small] = (erf - 2.0 * rl / (se * math.sqrt(math.pi)) * np.exp(-(rl * rl) / (se * se))) / rl ** 3
    return out


def fit_coeffs(rcut: float = 3.0, eps: float = 0.01, n_nodes: int = 4096,
               se: float | None = None) -> np.ndarray:
    """Constrained float64 least-squares fit; returns c[0..5] (float64)."""
    s_max = rcut * rcut
    k = np.arange(n_nodes)
    nodes = 0.5 * s_max * (1.0 - np.cos(math.pi * (k + 0.5) / n_nodes))
    g = gaussian_grid_force(nodes, se)
    # scale s to [0, 1] for conditioning: poly(s) = sum b_k (s/s_max)^k
    t = nodes / s_max
    A = np.vander(t, 6, increasing=True)
    # equality constraint at t = 1: sum b_k = (s_max + eps)^-1.5
    C = np.ones((1, 6))
    d = np.array([(s_max + eps) ** -1.5])
    # KKT system of the equality-constrained least-squares problem
    K = np.zeros((7, 7))
    K[:6, :6] = 2.0 * A.T @ A
    K[:6, 6:] = C.T
    K[6:, :6] = C
    rhs = np.concatenate([2.0 * A.T @ g, d])
    sol = np.linalg.solve(K, rhs)
    b = sol[:6]
    return b / s_max ** np.arange(6)


def default_coeffs(rcut: float = 3.0, eps: float = 0.01) -> np.ndarray:
    """The default coefficients as float32 (the precision the kernel uses)."""
    return fit_coeffs(rcut, eps).astype(np.float32)


def fit_report(rcut: float = 3.0, eps: float = 0.01) -> dict:
    c = fit_coeffs(rcut, eps)
    s = np.linspace(0.0, rcut * rcut, 2001)
    g = gaussian_grid_force(s)
    p = np.polynomial.polynomial.polyval(s, c)
    return {
        "coeffs": c.tolist(),
        "max_abs_residual": float(np.max(np.abs(p - g))),
        "max_rel_residual_vs_g0": float(np.max(np.abs(p - g)) / g[0]),
        "f_sr_at_cutoff": float((rcut * rcut + eps) ** -1.5 - np.polynomial.polynomial.polyval(rcut * rcut, c)),
    }


if __name__ == "__main__":
    import json
    print(json.dumps(fit_report(), indent=1))
