"""Pins of the oracle's short-range sub-cycles (oracle/sks.py) against what
the mathematics of the paper's symmetric stream-kick-stream map (Eq. 6)
fixes, on the CPU.

* one sub-cycle from rest: the half-streams do nothing, the kick uses the
  force at the starting point, so v_1 = h a(x_0) and x_1 = x_0 + (h^2/2) a(x_0)
  exactly (a kick-stream-kick or stream-first-by-h map gives other values);
* a free particle streams by exactly h v per sub-cycle, wrapped into [0, L);
* time reversibility: n_c sub-cycles with h, then n_c with -h, return to the
  start to float64 rounding (the map is symmetric);
* second order: on a circular two-body orbit of the softened force (c = 0,
  closed-form angular velocity) the position error after a fixed time falls
  four-fold when h halves;
* the energy is the closed-form kinetic plus pair potential energy, and it
  stays constant on the circular orbit.

Each check takes the sub-cycle module as an argument so that the mutation
test can run it on planted mistakes.
"""

import math

import numpy as np
import pytest

from oracle import sks as sks_mod
from synth import default_coeffs

EPS, RC = 0.01, 3.0


def _circular_pair(r=1.0, eps=EPS, L=16.0):
    """Two unit masses a distance r apart on a circular orbit about (L/2, L/2, L/2)
    in the plane z = L/2 under f(s) = (s + eps)^-3/2 (c = 0).  Returns
    (x0, v0, omega): each particle has centripetal acceleration f(r^2) r, so
    v = r sqrt(f / 2) and omega = sqrt(2 f)."""
    f = (r * r + eps) ** -1.5
    v = r * math.sqrt(f / 2.0)
    c = L / 2.0
    x0 = np.array([[c - r / 2, c, c], [c + r / 2, c, c]])
    v0 = np.array([[0.0, -v, 0.0], [0.0, v, 0.0]])
    return x0, v0, math.sqrt(2.0 * f)


def check_one_subcycle_from_rest(sks=sks_mod):
    c = np.zeros(6)
    r, m1, m2 = 1.3, 1.0, 2.0
    x0 = np.array([[5.0, 6.0, 7.0], [5.0 + r, 6.0, 7.0]])
    h = 0.05
    x1, v1, _ = sks.subcycles(x0, np.zeros((2, 3)), np.array([m1, m2]), 16.0, EPS, RC, c, h, 1)
    f = (r * r + EPS) ** -1.5
    a0 = np.array([[m2 * f * r, 0.0, 0.0], [-m1 * f * r, 0.0, 0.0]])  # attractive, a_i = m_j f d_ij
    assert np.allclose(v1, h * a0, rtol=1e-14, atol=0.0)
    assert np.allclose(x1, x0 + 0.5 * h * h * a0, rtol=0.0, atol=1e-14)


def check_free_particle_streams_and_wraps(sks=sks_mod):
    c = default_coeffs(RC, EPS).astype(np.float64)
    L = 8.0
    x0 = np.array([[7.9, 0.05, 4.0], [2.0, 2.0, 2.0 + RC + 1.0]])  # beyond the cutoff of each other
    v0 = np.array([[1.0, -2.0, 0.5], [0.0, 0.0, 0.0]])
    h = 0.125
    for n_c in (1, 4):  # one sub-cycle: particle 0 crosses x = L in the second half-stream
        x, v, _ = sks.subcycles(x0, v0, np.ones(2), L, EPS, RC, c, h, n_c)
        assert np.array_equal(v, v0)
        assert np.allclose(x, np.mod(x0 + n_c * h * v0, L), rtol=0.0, atol=1e-13)
        assert np.all((x >= 0.0) & (x < L))


def check_time_reversible(sks=sks_mod):
    c = default_coeffs(RC, EPS).astype(np.float64)
    rng = np.random.default_rng(21)
    N, L = 48, 8.0
    x0 = rng.random((N, 3)) * L
    v0 = rng.normal(0.0, 0.3, (N, 3))
    m = rng.uniform(0.5, 2.0, N)
    h, n_c = 0.01, 12
    x1, v1, _ = sks.subcycles(x0, v0, m, L, EPS, RC, c, h, n_c)
    assert np.max(np.abs(x1 - x0)) > 1e-3  # it did move
    x2, v2, _ = sks.subcycles(x1, v1, m, L, EPS, RC, c, -h, n_c)
    d = x2 - x0
    d -= L * np.round(d / L)
    assert np.max(np.abs(d)) < 1e-11
    assert np.max(np.abs(v2 - v0)) < 1e-11


def _orbit_error(sks, h, T):
    x0, v0, om = _circular_pair()
    n_c = int(round(T / h))
    x, v, hist = sks.subcycles(x0, v0, np.ones(2), 16.0, EPS, RC, np.zeros(6), h, n_c)
    t = n_c * h
    c = 8.0
    exact = np.array([[c - 0.5 * math.cos(om * t), c - 0.5 * math.sin(om * t), c],
                      [c + 0.5 * math.cos(om * t), c + 0.5 * math.sin(om * t), c]])
    return float(np.max(np.abs(x - exact))), hist


def check_second_order_on_circular_orbit(sks=sks_mod):
    e1, _ = _orbit_error(sks, 0.02, 2.0)
    e2, _ = _orbit_error(sks, 0.01, 2.0)
    assert 1e-7 < e2 < e1 < 1e-3
    assert 3.6 < e1 / e2 < 4.4, (e1, e2)


def check_energy_closed_form_and_conservation(sks=sks_mod):
    # closed form: kinetic sum m v^2 / 2, potential m_1 m_2 V(s) (each pair once),
    # V(s) = (r_c^2 + eps)^-1/2 - (s + eps)^-1/2 for c = 0
    x = np.array([[1.0, 1.0, 1.0], [1.0, 2.5, 1.0]])
    v = np.array([[0.5, 0.0, -1.0], [0.0, 2.0, 0.0]])
    m = np.array([1.5, 0.5])
    kin, pot = sks.energy(x, v, m, 16.0, EPS, RC, np.zeros(6))
    assert kin == pytest.approx(0.5 * (1.5 * 1.25 + 0.5 * 4.0), rel=1e-15)
    s = 1.5 ** 2
    assert pot == pytest.approx(1.5 * 0.5 * ((RC * RC + EPS) ** -0.5 - (s + EPS) ** -0.5), rel=1e-14)
    # circular orbit: kinetic and potential both constant
    x0, v0, _ = _circular_pair()
    k0, p0 = sks.energy(x0, v0, np.ones(2), 16.0, EPS, RC, np.zeros(6))
    _, hist = _orbit_error(sks, 0.01, 2.0)
    e = np.array([k + p for k, p in hist])
    assert np.max(np.abs(e - (k0 + p0))) < 1e-5 * abs(p0)


SKS_CHECKS = [check_one_subcycle_from_rest, check_free_particle_streams_and_wraps, check_time_reversible,
              check_second_order_on_circular_orbit, check_energy_closed_form_and_conservation]


@pytest.mark.parametrize("check", SKS_CHECKS, ids=lambda f: f.__name__)
def test_sks_oracle(check):
    check()
