"""Pins of the float64 CPU oracle against closed forms, invariants, library
routines and brute force (no GPU).

Each test is chosen so that a plausible slip in the oracle -- a dropped
softening, a wrong sign of d, a swapped mass, a wrong polynomial index, a
missing periodic image, an unstable sort, a missing neighbour cell -- fails.
"""

import json
import math
import os

import numpy as np
import pytest

import oracle
from synth import default_coeffs, fit_coeffs, gaussian_grid_force, uniform_box
from synth import gridfit

HERE = os.path.dirname(os.path.abspath(__file__))
EPS = 0.01
RC = 3.0


def _two(x1, x2, m1=1.0, m2=1.0, L=16.0):
    x = np.array([x1[0], x2[0]])
    y = np.array([x1[1], x2[1]])
    z = np.array([x1[2], x2[2]])
    return x, y, z, np.array([m1, m2]), L


# --------------------------------------------------------------------------
# force law
# --------------------------------------------------------------------------

def test_softened_newton_closed_form():
    """c = 0: the law is softened Newtonian gravity truncated at r_c.

    Textbook: a_1 = m_2 d / (r^2 + eps)^(3/2), d = x_2 - x_1 (attractive)."""
    c = np.zeros(6)
    for r, eps, m2 in [(1.0, 0.01, 2.5), (0.3, 0.5, 1.0), (2.9, 1e-6, 0.7)]:
        x, y, z, m, L = _two((5.0, 5.0, 5.0), (5.0 + r, 5.0, 5.0), m1=1.3, m2=m2)
        a = oracle.sr_force(x, y, z, m, L, eps, RC, c)
        expect = m2 * r / (r * r + eps) ** 1.5
        assert a[0, 0] == pytest.approx(expect, rel=1e-14)
        assert a[0, 1] == 0.0 and a[0, 2] == 0.0
        # particle 2 is pulled back towards particle 1 by m_1 (not m_2)
        assert a[1, 0] == pytest.approx(-1.3 * r / (r * r + eps) ** 1.5, rel=1e-14)


def test_newton_limit_inverse_square():
    """eps -> 0, c = 0: |a| = m / r^2 (Newton)."""
    c = np.zeros(6)
    r = 1.7
    x, y, z, m, L = _two((1.0, 2.0, 3.0), (1.0, 2.0 + r, 3.0), m2=3.0)
    a = oracle.sr_force(x, y, z, m, L, 1e-300, RC, c)
    assert np.linalg.norm(a[0]) == pytest.approx(3.0 / r ** 2, rel=1e-12)


def test_polynomial_term_matches_numpy_polyval():
    """The subtracted grid term equals numpy's polynomial evaluation.

    Uses a random non-symmetric coefficient set so a wrong power or index
    shows up; the Newtonian part is removed by differencing against c = 0."""
    rng = np.random.default_rng(11)
    c = rng.normal(size=6) * np.array([1, 0.3, 0.1, 0.03, 0.01, 0.003])
    for r in [0.4, 1.1, 2.2, 2.95]:
        s = r * r
        x, y, z, m, L = _two((3.0, 3.0, 3.0), (3.0, 3.0, 3.0 + r), m2=1.0)
        a_c = oracle.sr_force(x, y, z, m, L, EPS, RC, c)[0, 2]
        a_0 = oracle.sr_force(x, y, z, m, L, EPS, RC, np.zeros(6))[0, 2]
        assert (a_0 - a_c) / r == pytest.approx(np.polynomial.polynomial.polyval(s, c), rel=1e-12,
                                                abs=1e-14)
        # and the scalar helpers agree with the same definitions
        assert oracle.fsr(s, EPS, c) == pytest.approx(a_c / r, rel=1e-12)
        dnum = (oracle.fsr(s + 1e-6, EPS, c) - oracle.fsr(s - 1e-6, EPS, c)) / 2e-6
        assert oracle.dfsr(s, EPS, c) == pytest.approx(dnum, rel=1e-6)


def test_cutoff_is_exact_zero_and_strict():
    c = default_coeffs().astype(np.float64)
    # beyond the cutoff, and exactly at it (strict s < r_c^2)
    for r in [3.0, 3.0001, 5.0, 7.9]:
        x, y, z, m, L = _two((4.0, 4.0, 4.0), (4.0 + r, 4.0, 4.0))
        a = oracle.sr_force(x, y, z, m, L, EPS, RC, c)
        assert np.all(a == 0.0)
    # isolated particle: exactly zero
    a = oracle.sr_force(np.array([1.0]), np.array([1.0]), np.array([1.0]), np.array([1.0]),
                        16.0, EPS, RC, c)
    assert np.all(a == 0.0)


def test_periodic_image_across_boundary():
    """x = 0.5 and x = L - 0.5 are 1 apart through the boundary."""
    c = default_coeffs().astype(np.float64)
    L = 16.0
    x, y, z, m, _ = _two((0.5, 8.0, 8.0), (L - 0.5, 8.0, 8.0))
    a = oracle.sr_force(x, y, z, m, L, EPS, RC, c)
    f1 = oracle.fsr(1.0, EPS, c)
    assert f1 > 0
    # particle 0 is pulled towards -x (through the boundary), particle 1 towards +x
    assert a[0, 0] == pytest.approx(-f1, rel=1e-14)
    assert a[1, 0] == pytest.approx(+f1, rel=1e-14)


def test_newton_third_law_and_translation_invariance():
    c = default_coeffs().astype(np.float64)
    w = uniform_box(600, 8.0, seed=7)
    rng = np.random.default_rng(3)
    m = rng.uniform(0.5, 2.0, w.N)
    a = oracle.sr_force(w.x, w.y, w.z, m, 8.0, EPS, RC, c)
    mom = (m[:, None] * a).sum(0)
    scale = (m[:, None] * np.abs(a)).sum()
    assert np.all(np.abs(mom) < 1e-12 * scale)
    shift = rng.uniform(0, 8.0, 3)
    xs = np.mod(w.x.astype(np.float64) + shift[0], 8.0)
    ys = np.mod(w.y.astype(np.float64) + shift[1], 8.0)
    zs = np.mod(w.z.astype(np.float64) + shift[2], 8.0)
    a2 = oracle.sr_force(xs, ys, zs, m, 8.0, EPS, RC, c)
    assert np.max(np.abs(a2 - a)) < 1e-10 * np.max(np.abs(a))


def test_superposition_and_mass_linearity():
    c = default_coeffs().astype(np.float64)
    pts = np.array([[4.0, 4.0, 4.0], [5.0, 4.5, 4.2], [3.1, 3.3, 5.0]])
    m = np.array([1.0, 2.0, 0.5])
    a = oracle.sr_force(pts[:, 0], pts[:, 1], pts[:, 2], m, 12.0, EPS, RC, c)
    a01 = oracle.sr_force(pts[:2, 0], pts[:2, 1], pts[:2, 2], m[:2], 12.0, EPS, RC, c)
    a02 = oracle.sr_force(pts[[0, 2], 0], pts[[0, 2], 1], pts[[0, 2], 2], m[[0, 2]], 12.0, EPS,
                          RC, c)
    assert np.allclose(a[0], a01[0] + a02[0], rtol=1e-14, atol=0)


def test_perfect_lattice_has_zero_force():
    """Every particle of a perfect periodic lattice feels no net force."""
    c = default_coeffs().astype(np.float64)
    g = np.arange(8) + 0.5
    gz, gy, gx = np.meshgrid(g, g, g, indexing="ij")
    a = oracle.sr_force(gx.ravel(), gy.ravel(), gz.ravel(), np.ones(512), 8.0, EPS, RC, c)
    assert np.max(np.abs(a)) < 1e-12


def test_brute_force_small_against_independent_numpy():
    """Tiny N: a dense numpy evaluation (minimum image by rounding, masked sum)."""
    c = default_coeffs().astype(np.float64)
    rng = np.random.default_rng(5)
    N, L = 40, 7.0
    p = rng.random((N, 3)) * L
    m = rng.uniform(0.5, 1.5, N)
    a = oracle.sr_force(p[:, 0], p[:, 1], p[:, 2], m, L, EPS, RC, c)
    d = p[None, :, :] - p[:, None, :]
    d -= L * np.round(d / L)
    s = (d * d).sum(-1)
    mask = (s < RC * RC) & ~np.eye(N, dtype=bool)
    f = np.where(mask, (s + EPS) ** -1.5 - np.polynomial.polynomial.polyval(s, c), 0.0)
    ref = (m[None, :, None] * f[..., None] * d).sum(1)
    assert np.allclose(a, ref, rtol=1e-12, atol=1e-12)
    assert oracle.pair_count(p[:, 0], p[:, 1], p[:, 2], L, RC) == int(mask.sum())


def test_potential_closed_form_and_cutoff():
    """c = 0: V(s) = (r_c^2 + eps)^-1/2 - (s + eps)^-1/2 (softened Newton, shifted
    to vanish at r_c); and V(r_c^2) = 0 for any coefficients."""
    for r, eps in [(0.5, 0.01), (2.0, 0.3)]:
        x, y, z, m, L = _two((4.0, 4.0, 4.0), (4.0 + r, 4.0, 4.0), m1=1.0, m2=2.0)
        phi = oracle.sr_potential(x, y, z, m, L, eps, RC, np.zeros(6))
        expect = (RC * RC + eps) ** -0.5 - (r * r + eps) ** -0.5
        assert phi[0] == pytest.approx(2.0 * expect, rel=1e-13)
        assert phi[1] == pytest.approx(expect, rel=1e-13)
    rng = np.random.default_rng(8)
    assert abs(oracle.pair_potential(RC * RC, EPS, RC, rng.normal(size=6))) < 1e-13


def test_force_is_minus_gradient_of_potential_energy():
    """E = sum_i m_i phi_i / 2 and -dE/dx_i = m_i a_i (finite differences):
    ties the potential to the force law without retyping either."""
    c = default_coeffs().astype(np.float64)
    rng = np.random.default_rng(9)
    L, N = 7.0, 60
    while True:
        p = rng.random((N, 3)) * L
        if _pairs_clear_of_cutoff(p, L, 1e-3):
            break
    m = rng.uniform(0.5, 1.5, N)

    def E(pp):
        return 0.5 * float(np.sum(m * oracle.sr_potential(pp[:, 0], pp[:, 1], pp[:, 2], m, L, EPS, RC, c)))

    a = oracle.sr_force(p[:, 0], p[:, 1], p[:, 2], m, L, EPS, RC, c)
    h = 1e-6
    for i in [0, 13, 44]:
        for k in range(3):
            pp, pm = p.copy(), p.copy()
            pp[i, k] += h
            pm[i, k] -= h
            g = (E(pp) - E(pm)) / (2 * h)
            assert -g == pytest.approx(m[i] * a[i, k], rel=1e-6, abs=1e-8)


# --------------------------------------------------------------------------
# adjoint
# --------------------------------------------------------------------------

def _pairs_clear_of_cutoff(p, L, margin):
    d = p[None] - p[:, None]
    d -= L * np.round(d / L)
    r = np.sqrt((d * d).sum(-1))
    return np.all(np.abs(r - RC) > margin)


def test_adjoint_against_finite_differences():
    c = default_coeffs().astype(np.float64)
    rng = np.random.default_rng(21)
    L, N = 6.5, 48
    while True:
        p = rng.random((N, 3)) * L
        if _pairs_clear_of_cutoff(p, L, 1e-3):
            break
    m = rng.uniform(0.5, 1.5, N)
    lam = rng.normal(size=(N, 3))
    gx, gm = oracle.sr_force_adjoint(p[:, 0], p[:, 1], p[:, 2], m, L, EPS, RC, c, lam)

    def J(pp, mm):
        a = oracle.sr_force(pp[:, 0], pp[:, 1], pp[:, 2], mm, L, EPS, RC, c)
        return float((lam * a).sum())

    h = 1e-6
    for i in [0, 7, 31]:
        for k in range(3):
            pp, pm = p.copy(), p.copy()
            pp[i, k] += h
            pm[i, k] -= h
            fd = (J(pp, m) - J(pm, m)) / (2 * h)
            assert gx[i, k] == pytest.approx(fd, rel=1e-6, abs=1e-8)
        mp, mm = m.copy(), m.copy()
        mp[i] += h
        mm[i] -= h
        fd = (J(p, mp) - J(p, mm)) / (2 * h)
        assert gm[i] == pytest.approx(fd, rel=1e-6, abs=1e-8)


def test_adjoint_against_torch_float64_autograd():
    """Independent library check: float64 autograd of a dense expression."""
    torch = pytest.importorskip("torch")
    c = default_coeffs().astype(np.float64)
    rng = np.random.default_rng(22)
    L, N = 7.0, 96
    p = rng.random((N, 3)) * L
    m = rng.uniform(0.5, 1.5, N)
    lam = rng.normal(size=(N, 3))
    gx, gm = oracle.sr_force_adjoint(p[:, 0], p[:, 1], p[:, 2], m, L, EPS, RC, c, lam)

    P = torch.tensor(p, dtype=torch.float64, requires_grad=True)
    M = torch.tensor(m, dtype=torch.float64, requires_grad=True)
    d = P[None, :, :] - P[:, None, :]
    d = d - L * torch.round(d.detach() / L)
    s = (d * d).sum(-1)
    mask = (s < RC * RC) & ~torch.eye(N, dtype=torch.bool)
    ss = torch.where(mask, s, torch.ones_like(s))
    poly = sum(float(c[k]) * ss ** k for k in range(6))
    f = torch.where(mask, (ss + EPS) ** -1.5 - poly, torch.zeros_like(s))
    a = (M[None, :, None] * f[..., None] * d).sum(1)
    (a * torch.tensor(lam)).sum().backward()
    assert np.allclose(gx, P.grad.numpy(), rtol=1e-10, atol=1e-10)
    assert np.allclose(gm, M.grad.numpy(), rtol=1e-10, atol=1e-10)


def test_adjoint_as_one_antisymmetric_sum():
    """Without dL/dm the gradient is one vector sum per particle: with
    mu_ij = m_i lam_j - m_j lam_i and J(d) = f I + 2 f' d d^T, the pair adds
    w_ij = J(d_ij) mu_ij to dL/dx_i, and w_ji = -w_ij (the form the GPU adjoints
    sum; equal masses: m sum_j J(d_ij) (lam_j - lam_i)).  Dense numpy float64
    against the oracle's adjoint."""
    c = default_coeffs().astype(np.float64)
    rng = np.random.default_rng(23)
    L, N = 7.0, 80
    p = rng.random((N, 3)) * L
    lam = rng.normal(size=(N, 3))
    d = p[None, :, :] - p[:, None, :]  # d[i, j] = x_j - x_i, minimal image
    d -= L * np.round(d / L)
    s = (d * d).sum(-1)
    mask = (s < RC * RC) & ~np.eye(N, dtype=bool)
    f = np.where(mask, (s + EPS) ** -1.5 - np.polyval(c[::-1], s), 0.0)
    dc = np.arange(1, 6) * c[1:]
    fp2 = np.where(mask, 2.0 * (-1.5 * (s + EPS) ** -2.5 - np.polyval(dc[::-1], s)), 0.0)
    for m in (rng.uniform(0.5, 1.5, N), np.full(N, 0.37)):
        mu = m[:, None, None] * lam[None, :, :] - m[None, :, None] * lam[:, None, :]
        w = f[..., None] * mu + (fp2 * (d * mu).sum(-1))[..., None] * d
        assert np.allclose(w, -w.transpose(1, 0, 2), rtol=0, atol=1e-12)
        gx, _ = oracle.sr_force_adjoint(p[:, 0], p[:, 1], p[:, 2], m, L, EPS, RC, c, lam)
        assert np.allclose(w.sum(1), gx, rtol=1e-10, atol=1e-10)
    dl = lam[None, :, :] - lam[:, None, :]
    we = f[..., None] * dl + (fp2 * (d * dl).sum(-1))[..., None] * d
    assert np.allclose(0.37 * we.sum(1), gx, rtol=1e-10, atol=1e-10)


def test_trajectory_gradient_against_finite_differences():
    from oracle import diff
    c = default_coeffs().astype(np.float64)
    rng = np.random.default_rng(23)
    L, N = 7.0, 40
    while True:
        x0 = rng.random((N, 3)) * L
        if _pairs_clear_of_cutoff(x0, L, 2e-2):
            break
    v0 = rng.normal(scale=0.3, size=(N, 3))
    m = rng.uniform(0.5, 1.5, N)
    w = rng.normal(size=(N, 3))
    dt, steps = 0.01, 4
    gx, gv, gm = diff.gradient(x0, v0, m, L, EPS, RC, c, dt, steps, w)
    h = 1e-5
    for (i, k) in [(0, 0), (5, 1), (17, 2)]:
        fd = diff.finite_difference(x0, v0, m, L, EPS, RC, c, dt, steps, w, "x", (i, k), h)
        assert gx[i, k] == pytest.approx(fd, rel=1e-6, abs=1e-9)
        fd = diff.finite_difference(x0, v0, m, L, EPS, RC, c, dt, steps, w, "v", (i, k), h)
        assert gv[i, k] == pytest.approx(fd, rel=1e-6, abs=1e-9)
    for i in [3, 11]:
        fd = diff.finite_difference(x0, v0, m, L, EPS, RC, c, dt, steps, w, "m", i, h)
        assert gm[i] == pytest.approx(fd, rel=1e-6, abs=1e-9)


def test_kick_drift_exact_on_dyadic_values():
    v = np.array([[0.5, -0.25, 1.0]])
    a = np.array([[2.0, 4.0, -8.0]])
    x = np.array([[1.0, 2.0, 3.0]])
    v2, x2 = oracle.kick_drift(v, a, 0.125, x, 0.5)
    assert np.array_equal(v2, [[0.75, 0.25, 0.0]])
    assert np.array_equal(x2, [[1.375, 2.125, 3.0]])


# --------------------------------------------------------------------------
# binning, lists, tasks
# --------------------------------------------------------------------------

def _wrap_f32_numpy(x, L):
    """The binning's float32 wrap, restated with numpy float32 vector ops."""
    x = x.astype(np.float32)
    L = np.float32(L)
    q = np.floor(x / L)
    xw = x - q * L
    xw = np.where(xw < 0, xw + L, xw)
    xw = np.where(xw >= L, xw - L, xw)
    return xw.astype(np.float32)


def test_binning_invariants_and_numpy_restatement():
    rng = np.random.default_rng(31)
    L = np.float32(17.3)
    N = 3000
    x = (rng.random(N) * 3 * L - L).astype(np.float32)  # outside [0, L) too
    y = (rng.random(N) * L).astype(np.float32)
    z = (rng.normal(size=N) * 5).astype(np.float32)
    x[:4] = [0.0, -0.0, L, np.nextafter(L, np.float32(0))]
    x[4] = np.float32(-1e-9)
    m = rng.uniform(0.5, 2, N).astype(np.float32)
    b = oracle.bin_volume(x, y, z, m, float(L), 3.0)
    n, w, iw = b["n"], b["w"], b["inv_w"]
    assert n == 5 and w == np.float32(L / np.float32(5)) and iw == np.float32(np.float32(5) / L)
    cs, perm, s4 = b["cell_start"], b["perm"], b["sorted4"]
    assert cs[0] == 0 and cs[-1] == N and np.all(np.diff(cs) >= 0)
    assert np.array_equal(np.sort(perm), np.arange(N))
    # stable: ascending original index within each cell
    for c in range(n ** 3):
        seg = perm[cs[c]:cs[c + 1]]
        assert np.all(np.diff(seg) > 0)
        assert np.all(b["cell_of"][seg] == c)
    # numpy float32 restatement of the cell definition, bit for bit
    cells = []
    wr = []
    for arr in (x, y, z):
        xw = _wrap_f32_numpy(arr, L)
        assert np.all(xw >= 0) and np.all(xw < L)
        cc = np.minimum(np.floor(xw * iw).astype(np.int64), n - 1)
        cells.append(cc)
        wr.append(xw)
    cid = (cells[2] * n + cells[1]) * n + cells[0]
    assert np.array_equal(cid, b["cell_of"])
    for k, (cc, xw) in enumerate(zip(cells, wr)):
        ctr = ((cc.astype(np.float32) + np.float32(0.5)) * w).astype(np.float32)  # the cell centre
        o = (xw - ctr).astype(np.float32)
        assert np.array_equal(s4[:, k].view(np.int32), o[perm].view(np.int32))
    assert np.array_equal(s4[:, 3], m[perm])
    # offsets lie in the cell, [-w/2, w/2] about its centre (to float32 rounding),
    # and reproduce the position mod L
    assert np.all(s4[:, :3] > -0.5 * w - 1e-5) and np.all(s4[:, :3] < 0.5 * w + 1e-5)
    assert np.max(np.abs(s4[:, :3])) > 0.45 * w
    ccell = b["cell_of"][perm]
    org = (np.stack([ccell % n, (ccell // n) % n, ccell // (n * n)], 1) + 0.5) * np.float64(w)
    pos = np.stack([x, y, z], 1)[perm].astype(np.float64)
    diff = s4[:, :3].astype(np.float64) + org - pos
    diff -= np.float64(L) * np.round(diff / np.float64(L))
    assert np.max(np.abs(diff)) < 1e-5


def test_binning_with_displacements_keeps_float64_positions():
    """Displacement mode: the offset plus the cell centre reproduces the float64
    position x + d (mod L) to float32 precision of the offset (not of L), and
    the steps restate bit for bit in numpy float64."""
    rng = np.random.default_rng(32)
    L = np.float32(64.0)
    N = 4000
    x = (rng.random(N) * L).astype(np.float32)
    y = (rng.random(N) * L).astype(np.float32)
    z = (rng.random(N) * L).astype(np.float32)
    d = (rng.normal(size=(3, N)) * 1e-3).astype(np.float32)
    d[0, :3] = [-x[0] - np.float32(1e-6), np.float32(70.0), np.float32(-64.5)]
    # y + d = -1e-20: p - floor(p / L) L rounds to L itself, which the wrap's
    # correction step brings back to 0
    y[3], d[1, 3] = np.float32(0.0), np.float32(-1e-20)
    m = np.ones(N, np.float32)
    b = oracle.bin_volume(x, y, z, m, float(L), 3.0, disp=d)
    n, w, iw = b["n"], b["w"], b["inv_w"]
    s4, perm = b["sorted4"], b["perm"]
    pos = np.stack([x, y, z]).astype(np.float64) + d.astype(np.float64)
    for k in range(3):
        p = pos[k]
        q = np.floor(p / np.float64(L))
        pw = p - q * np.float64(L)
        pw = np.where(pw < 0, pw + np.float64(L), pw)
        pw = np.where(pw >= np.float64(L), pw - np.float64(L), pw)
        c = np.clip(np.floor(pw * np.float64(iw)).astype(np.int64), 0, n - 1)
        ctr = ((c.astype(np.float32) + np.float32(0.5)) * w).astype(np.float32)
        o = (pw - ctr.astype(np.float64)).astype(np.float32)
        assert np.array_equal(s4[:, k].view(np.int32), o[perm].view(np.int32))
        err = (o.astype(np.float64) + ctr - pw)
        assert np.max(np.abs(err)) <= 0.5 * np.spacing(np.float32(0.5 * w))
    cid = b["cell_of"]
    assert np.all(np.diff(cid[perm]) >= 0)


@pytest.mark.parametrize("L,cell_min,rcut", [(16.0, 3.0, 3.0), (10.0, 2.0, 3.0), (9.0, 3.0, 3.0),
                                             (13.0, 1.4, 3.0)])
def test_lists_cover_every_pair_within_cutoff(L, cell_min, rcut):
    """Brute force: every pair closer than r_c is in a listed (cell, image)."""
    rng = np.random.default_rng(41)
    N = 900
    p = (rng.random((N, 3)) * L).astype(np.float32)
    m = np.ones(N, np.float32)
    b = oracle.bin_volume(p[:, 0], p[:, 1], p[:, 2], m, L, cell_min)
    n, w = b["n"], b["w"]
    off, cell, shift = oracle.lists_volume(n, w, rcut)
    listed = set()
    for c in range(n ** 3):
        for e in range(off[c], off[c + 1]):
            listed.add((c, int(cell[e]), int(shift[e])))
    # neighbour entries are distinct and the box distance predicate is tight
    assert len(listed) == off[-1]
    R = oracle.reach(w, rcut)
    co = b["cell_of"]
    d = p[None].astype(np.float64) - p[:, None].astype(np.float64)
    img = np.round(d / L)
    d -= L * img
    s = (d * d).sum(-1)
    ii, jj = np.nonzero((s < rcut * rcut) & ~np.eye(N, dtype=bool))
    cx = lambda c: np.stack([c % n, (c // n) % n, c // (n * n)], -1)
    for i, j in zip(ii, jj):
        ci, cj = cx(co[i]), cx(co[j])
        delta = cj - ci
        # image that brings j next to i: the periodic offset of at most R cells
        sh = np.zeros(3, int)
        for a in range(3):
            if delta[a] > R:
                delta[a] -= n
                sh[a] = -1
            elif delta[a] < -R:
                delta[a] += n
                sh[a] = 1
        code = (sh[2] + 1) * 9 + (sh[1] + 1) * 3 + (sh[0] + 1)
        assert (int(co[i]), int(co[j]), code) in listed
    if w >= rcut:
        assert np.all(np.diff(off) == 27)


def _interval_gap_d2(a0, a1, b0, b1):
    """Squared distance between the closest points of two axis-aligned boxes
    [a0, a1] and [b0, b1] (float64 arrays of 3 per box, leading axes
    broadcast): the closest point of box a to box b's low corner, then the
    closest point of box b to that point."""
    pa = np.clip(b0, a0, a1)
    pb = np.clip(pa, b0, b1)
    return ((pb - pa) ** 2).sum(-1)


@pytest.mark.parametrize("L,cell_min,rcut", [(10.0, 2.0, 3.0), (9.0, 1.0, 3.0), (6.4, 0.375, 3.0),
                                             (16.0, 3.0, 3.0)])
def test_lists_are_exactly_the_cells_whose_boxes_come_closer_than_rc(L, cell_min, rcut):
    """Tightness: a neighbour (cell, image) is listed iff the two cell boxes
    have points closer than r_c.  The boxes are laid out from the mesh's cell
    width, the closest points found by projection, over a window one cell
    wider than the stencil.  Meshes: reach 2, reach 3 with w = 1 (offsets
    (3, 3, 2) leave gaps (2, 2, 1) w, exactly r_c, so a non-strict test would
    list them), reach 8, and the 27-cell case."""
    n, w, _ = oracle.mesh(L, cell_min)
    R = oracle.reach(w, rcut)
    off, cell, shift = oracle.lists_volume(n, w, rcut)
    W = float(w)
    win = np.array([(dx, dy, dz) for dz in range(-R - 1, R + 2) for dy in range(-R - 1, R + 2)
                    for dx in range(-R - 1, R + 2)], np.int64)
    rng = np.random.default_rng(3)
    cells = {0, n ** 3 - 1, (n // 2) * (n * n + n + 1)} | set(rng.integers(0, n ** 3, 5).tolist())
    for c in sorted(cells):
        cc = np.array([c % n, (c // n) % n, c // (n * n)], np.int64)
        got = set()
        for e in range(off[c], off[c + 1]):
            p = int(cell[e])
            pc = np.array([p % n, (p // n) % n, p // (n * n)], np.int64)
            code = int(shift[e])
            sh = np.array([code % 3 - 1, (code // 3) % 3 - 1, code // 9 - 1], np.int64)
            got.add(tuple((pc + sh * n - cc).tolist()))
        assert len(got) == off[c + 1] - off[c]
        lo_a = cc * W
        lo_b = (cc + win) * W
        d2 = _interval_gap_d2(lo_a, lo_a + W, lo_b, lo_b + W)
        expect = {tuple(d.tolist()) for d in win[d2 < rcut * rcut]}
        assert got == expect, (c, sorted(got ^ expect)[:6])
    if (L, cell_min) == (9.0, 1.0):
        assert (3, 3, 2) not in got and (3, 3, 1) in got


def test_lists_reject_too_coarse_mesh():
    with pytest.raises(ValueError):
        oracle.lists_volume(4, 1.0, 3.0)   # R = 3 needs n >= 7


def test_tasks_partition_each_cell():
    w = uniform_box(2000, 12.0, seed=9)
    b = oracle.bin_volume(w.x, w.y, w.z, w.m, 12.0, 3.0)
    t = oracle.tasks(b["cell_start"], 7)
    assert np.all(t[:, 2] - t[:, 1] <= 7) and np.all(t[:, 2] > t[:, 1])
    assert t[0, 1] == 0 and t[-1, 2] == 2000 and np.all(t[1:, 1] == t[:-1, 2])
    for c, s, e in t:
        assert b["cell_start"][c] <= s < e <= b["cell_start"][c + 1]


# --------------------------------------------------------------------------
# RCB fat-leaf tree (Sec. III) and its leaf lists
# --------------------------------------------------------------------------

def test_rcb_hand_worked_examples():
    """Small trees worked out by hand from the rule (centre-of-mass split
    along the longest side, left iff q <= floor(mean q), stable halves).
    L = 64: q = 32768 x exactly for these positions."""
    one = np.ones(6, np.float32)
    x = np.array([1, 9, 2, 8, 3, 10], np.float32)
    y = np.array([0, 0, 0, 1, 0, 0], np.float32)
    z = np.zeros(6, np.float32)
    # root: x spans 9, mean 5.5 -> {0, 2, 4} | {1, 3, 5}; left: mean 2 -> {0, 2} | {4} (x = 2 goes
    # left: q <= split); right: x spans 2 > y's 1, mean 9 -> {1, 3} | {5}
    r = oracle.rcb_volume(x, y, z, one, 64.0, 2)
    assert r["perm"].tolist() == [0, 2, 4, 1, 3, 5]
    assert r["leaf_start"].tolist() == [0, 2, 3, 5, 6]
    assert (r["leaf_qbox"] // 32768).tolist() == [[1, 0, 0, 2, 0, 0], [3, 0, 0, 3, 0, 0],
                                                  [8, 0, 0, 9, 1, 0], [10, 0, 0, 10, 0, 0]]
    # depth cap 1: only the root splits
    r = oracle.rcb_volume(x, y, z, one, 64.0, 2, max_depth=1)
    assert r["leaf_start"].tolist() == [0, 3, 6]
    # the longest side decides the axis: y spans 6 > x's 2
    x2 = np.array([1, 2, 3, 1, 2, 3], np.float32)
    y2 = np.array([0, 6, 1, 5, 2, 4], np.float32)
    r = oracle.rcb_volume(x2, y2, z, one, 64.0, 3)
    assert r["perm"].tolist() == [0, 2, 4, 1, 3, 5]  # mean y 3: {0, 2, 4} (y 0, 1, 2) | {1, 3, 5}
    # a mean between grid points is floored: q = q0 + (0, 1, 1) has mean q0 + 2/3, so only the
    # first particle goes left (rounding up would keep all three together)
    u = np.float32(1.0 / 32768)
    x3 = np.array([10.0, 10.0 + u, 10.0 + u], np.float32)
    r = oracle.rcb_volume(x3, z[:3], z[:3], one[:3], 64.0, 1)
    assert r["leaf_start"].tolist() == [0, 1, 2, 3]
    # coincident particles: halves by position, cnt / 2 to the left
    c3 = np.full(3, 7.0, np.float32)
    r = oracle.rcb_volume(c3, c3, c3, one[:3], 64.0, 1)
    assert r["perm"].tolist() == [0, 1, 2] and r["leaf_start"].tolist() == [0, 1, 2, 3]


def test_rcb_regular_lattice_is_bit_interleaved():
    """On a 4^3 lattice every centre of mass is a midpoint, so each split halves
    the group and the axis cycles x, y, z (ties go to the lowest axis): the
    leaf order is the bit-interleaved (Morton) order with x most significant."""
    L = 16.0
    g = np.arange(4)
    ix, iy, iz = [a.reshape(-1) for a in np.meshgrid(g, g, g, indexing="ij")]
    order = np.random.default_rng(5).permutation(64)
    ix, iy, iz = ix[order], iy[order], iz[order]
    x, y, z = [(4 * a + 1).astype(np.float32) for a in (ix, iy, iz)]
    m = np.ones(64, np.float32)
    key = lambda a, b, c: (a >> 1) * 32 + (b >> 1) * 16 + (c >> 1) * 8 + (a & 1) * 4 + (b & 1) * 2 + (c & 1)
    k = key(ix, iy, iz)
    r = oracle.rcb_volume(x, y, z, m, L, 1)
    assert r["n_leaves"] == 64 and np.array_equal(k[r["perm"]], np.arange(64))
    r = oracle.rcb_volume(x, y, z, m, L, 8)
    assert r["leaf_start"].tolist() == list(range(0, 65, 8))
    octant = k[r["perm"]] // 8
    assert np.array_equal(octant, np.repeat(np.arange(8), 8))
    for l in range(8):  # stable: input order within each leaf
        assert np.all(np.diff(r["perm"][8 * l:8 * l + 8]) > 0)


def _quant21_numpy(xw, L):
    return np.minimum(np.floor(xw.astype(np.float64) * (2.0 ** 21 / np.float64(L))), 2 ** 21 - 1).astype(np.int64)


def test_rcb_leaves_invariants_on_clustered_particles():
    from synth.workloads import clustered_box
    w = clustered_box(24, 3, seed=17)
    L = float(w.L[0])
    for leaf_max in (1, 7, 32, 64):
        r = oracle.rcb_volume(w.x, w.y, w.z, w.m, L, leaf_max)
        perm, ls, qb, s4 = r["perm"], r["leaf_start"], r["leaf_qbox"], r["sorted4"]
        assert np.array_equal(np.sort(perm), np.arange(w.N))
        sizes = np.diff(ls)
        assert ls[0] == 0 and ls[-1] == w.N and np.all(sizes >= 1) and np.all(sizes <= leaf_max)
        xw = [_wrap_f32_numpy(a, L) for a in (w.x, w.y, w.z)]
        q = np.stack([_quant21_numpy(a, L) for a in xw], 1)
        scale = L / 2.0 ** 21
        for l in range(r["n_leaves"]):
            idx = perm[ls[l]:ls[l + 1]]
            assert np.all(np.diff(idx) > 0)  # stable partitions keep input order
            assert np.array_equal(qb[l, :3], q[idx].min(0)) and np.array_equal(qb[l, 3:], q[idx].max(0))
            org = (qb[l, :3] * scale).astype(np.float32).astype(np.float64)
            for a in range(3):
                pos = s4[ls[l]:ls[l + 1], a].astype(np.float64) + org[a]
                assert np.max(np.abs(pos - xw[a][idx])) <= 2 * np.spacing(np.float32(L))
        assert np.array_equal(s4[:, 3], w.m[perm])
    # a group of more than leaf_max particles always splits in two non-empty halves,
    # so the leaves of one size bound nest in those of a larger one
    big = oracle.rcb_volume(w.x, w.y, w.z, w.m, L, 64)
    small = oracle.rcb_volume(w.x, w.y, w.z, w.m, L, 32)
    assert set(big["leaf_start"].tolist()) <= set(small["leaf_start"].tolist())
    for b, e in zip(big["leaf_start"][:-1], big["leaf_start"][1:]):
        assert np.array_equal(np.sort(big["perm"][b:e]), np.sort(small["perm"][b:e]))


@pytest.mark.parametrize("maker,leaf_max", [("uniform", 16), ("clustered", 24)])
def test_rcb_lists_cover_every_pair_within_cutoff(maker, leaf_max):
    """Brute force: every pair closer than r_c sits in a listed (leaf, leaf,
    image); the lists are symmetric, hold each leaf itself, and are in
    canonical order."""
    from synth.workloads import clustered_box
    w = uniform_box(1200, 12.0, seed=8) if maker == "uniform" else clustered_box(16, 2, seed=9)
    L = float(w.L[0])
    r = oracle.rcb_volume(w.x, w.y, w.z, w.m, L, leaf_max)
    off, leaf, shift = oracle.rcb_lists(r["leaf_qbox"], L, RC)
    nl = r["n_leaves"]
    listed = set()
    for i in range(nl):
        ent = list(zip(shift[off[i]:off[i + 1]].tolist(), leaf[off[i]:off[i + 1]].tolist()))
        assert ent == sorted(ent) and len(set(ent)) == len(ent)
        assert (13, i) in ent
        listed.update((i, j, c) for c, j in ent)
    assert all((j, i, 26 - c) in listed for i, j, c in listed)
    leaf_of = np.zeros(w.N, np.int64)
    for l in range(nl):
        leaf_of[r["perm"][r["leaf_start"][l]:r["leaf_start"][l + 1]]] = l
    p = np.stack([_wrap_f32_numpy(a, L) for a in (w.x, w.y, w.z)], 1).astype(np.float64)
    d = p[None] - p[:, None]          # d[i, j] = x_j - x_i
    img = -np.round(d / L)            # image s of j that lies next to i
    dd = d + L * img
    close = ((dd * dd).sum(-1) < RC * RC) & ~np.eye(w.N, dtype=bool)
    ii, jj = np.nonzero(close)
    sh = img[ii, jj].astype(int)
    code = (sh[:, 2] + 1) * 9 + (sh[:, 1] + 1) * 3 + (sh[:, 0] + 1)
    missing = [(a, b, c) for a, b, c in zip(leaf_of[ii], leaf_of[jj], code) if (a, b, c) not in listed]
    assert not missing, missing[:5]
    assert len(ii) > 1000


def _rcb_expected_lists(qbox, L, rcut):
    """Every (i, j, image code) whose leaf boxes, widened by one grid step on
    every side, have points closer than r_c (closest points by projection)."""
    q = np.asarray(qbox, np.float64)
    step = L / 2 ** 21
    lo = (q[:, :3] - 1) * step
    hi = (q[:, 3:] + 2) * step
    out = set()
    for code in range(27):
        sh = np.array([code % 3 - 1, (code // 3) % 3 - 1, code // 9 - 1], np.float64) * L
        d2 = _interval_gap_d2(lo[:, None], hi[:, None], lo[None] + sh, hi[None] + sh)
        ii, jj = np.nonzero(d2 < rcut * rcut)
        out.update(zip(ii.tolist(), jj.tolist(), [code] * len(ii)))
    return out


@pytest.mark.parametrize("maker,leaf_max", [("uniform", 16), ("clustered", 24)])
def test_rcb_lists_are_exactly_the_leaves_whose_widened_boxes_come_closer(maker, leaf_max):
    """Tightness of the leaf lists: (leaf j, image) is listed for leaf i iff
    the widened boxes have points closer than r_c, and nothing else is."""
    from synth.workloads import clustered_box
    w = uniform_box(1200, 12.0, seed=8) if maker == "uniform" else clustered_box(16, 2, seed=9)
    L = float(w.L[0])
    r = oracle.rcb_volume(w.x, w.y, w.z, w.m, L, leaf_max)
    off, leaf, shift = oracle.rcb_lists(r["leaf_qbox"], L, RC)
    got = set()
    for i in range(r["n_leaves"]):
        got.update((i, int(j), int(c)) for j, c in zip(leaf[off[i]:off[i + 1]], shift[off[i]:off[i + 1]]))
    assert len(got) == off[-1]
    assert got == _rcb_expected_lists(r["leaf_qbox"], L, RC)


def test_rcb_lists_cutoff_is_strict_on_exact_gaps():
    """Hand-made leaf boxes on a box of 16 (grid step 2^-17, exact in float64):
    leaf 1's widened box starts exactly r_c = 3 beyond leaf 0's, leaf 2's one
    step closer.  Only leaf 2 (and leaf 0 itself) may be listed for leaf 0,
    and leaf 0 may not be listed for leaf 1 (the same gap seen from the right:
    a box widened by more than one step on that side would list it)."""
    L = 16.0
    q0 = [0, 0, 0, 10, 10, 10]
    g = 3 * 2 ** 17 + 13  # widened gap: (g - 1) - (10 + 2) steps = 3 * 2^17 steps = 3.0
    q1 = [g, 0, 0, g + 10, 10, 10]
    q2 = [g - 1, 20, 0, g + 9, 30, 10]
    off, leaf, shift = oracle.rcb_lists(np.array([q0, q1, q2], np.int32), L, RC, targets=[0, 1])
    ent0 = set(zip(leaf[off[0]:off[1]].tolist(), shift[off[0]:off[1]].tolist()))
    ent1 = set(zip(leaf[off[1]:off[2]].tolist(), shift[off[1]:off[2]].tolist()))
    assert ent0 == {(0, 13), (2, 13)}
    assert ent1 == {(1, 13), (2, 13)}


# --------------------------------------------------------------------------
# grid-force fit (input generator of the coefficients)
# --------------------------------------------------------------------------

def test_gridfit_against_paper_constants_and_shell_theorem():
    from scipy import integrate
    consts = json.load(open(os.path.join(HERE, "golden", "paper_constants.json")))
    sig, ns = consts["filter_sigma"]["value"], consts["filter_ns"]["value"]
    se = gridfit.sigma_eff(sig, ns, 1.0)
    assert se == pytest.approx(math.sqrt(0.64 + 7.0 / 6.0))
    # shell theorem: g(r) r^3 = M(<r) of a 3-D Gaussian with per-axis std se/sqrt(2)
    sg = se / math.sqrt(2.0)
    rho = lambda r: 4 * math.pi * r * r * math.exp(-r * r / (2 * sg * sg)) / (2 * math.pi * sg * sg) ** 1.5
    for r in [0.2, 1.0, 2.5, 4.0]:
        M, _ = integrate.quad(rho, 0.0, r, epsabs=1e-14, epsrel=1e-12)
        assert gaussian_grid_force(np.array([r * r]), se)[0] * r ** 3 == pytest.approx(M, rel=1e-9)
    # small-r limit and large-r Newtonian asymptote
    assert gaussian_grid_force(np.array([0.0]), se)[0] == pytest.approx(
        4.0 / (3.0 * math.sqrt(math.pi) * se ** 3))
    assert gaussian_grid_force(np.array([400.0]), se)[0] * 20.0 ** 3 == pytest.approx(1.0, rel=1e-12)
    c = fit_coeffs(3.0, EPS)
    assert len(c) == consts["poly_degree"]["value"] + 1
    # continuity at the cutoff: f_SR(r_c^2) = 0
    assert abs((9.0 + EPS) ** -1.5 - np.polynomial.polynomial.polyval(9.0, c)) < 1e-15
    s = np.linspace(0, 9, 500)
    assert np.max(np.abs(np.polynomial.polynomial.polyval(s, c) - gaussian_grid_force(s, se))) < 1e-3
