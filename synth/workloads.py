"""Seeded particle sets standing in for the paper's cosmology workloads.

The paper runs on cosmological initial conditions and evolved density fields
(Sec. V) that are not available here.  These generators produce synthetic
sets with the same structure: a near-uniform density of one particle per grid
cell cubed (the paper's particle loading), optionally perturbed lattices
(Zel'dovich-style displacement of a lattice, as in cosmological initial
conditions), and NFW-profile halos that give the very uneven neighbour counts
of a clustered late-time field (Sec. II: the particle methods handle the
shortest scales, where clustering is strongest).

All random numbers come from numpy's PCG64 ``default_rng(seed)``, generated in
float64 and stored as float32, in the order written in each function.
"""

from __future__ import annotations

import dataclasses
import math

import numpy as np


@dataclasses.dataclass
class Workload:
    """One synthetic input.

    Particles of all volumes are concatenated; volume ``v`` owns the index
    range ``vol_off[v]:vol_off[v+1]`` and has periodic box side ``L[v]``.
    """

    name: str
    x: np.ndarray  # float32 [N]
    y: np.ndarray
    z: np.ndarray
    m: np.ndarray  # float32 [N]
    vx: np.ndarray  # float32 [N]
    vy: np.ndarray
    vz: np.ndarray
    L: np.ndarray  # float32 [V]
    vol_off: np.ndarray  # int64 [V+1]
    rcut: float = 3.0
    eps: float = 0.01
    cell_min: float = 3.0
    dt: float = 0.01
    extra: dict = dataclasses.field(default_factory=dict)

    @property
    def N(self) -> int:
        return int(self.vol_off[-1])

    @property
    def V(self) -> int:
        return int(self.L.shape[0])


def _wrap32(pos64: np.ndarray, L32: np.float32) -> np.ndarray:
    """Wrap float64 positions into [0, L) and store as float32 in [0, L)."""
    p = np.mod(pos64, float(L32)).astype(np.float32)
    p[p >= L32] = np.float32(0.0)
    p[p < 0] = np.float32(0.0)
    return p


def _single(name, pos, L32, **kw) -> Workload:
    n = pos.shape[0]
    x = _wrap32(pos[:, 0], L32)
    y = _wrap32(pos[:, 1], L32)
    z = _wrap32(pos[:, 2], L32)
    zeros = np.zeros(n, np.float32)
    return Workload(
        name=name, x=x, y=y, z=z, m=np.ones(n, np.float32),
        vx=zeros.copy(), vy=zeros.copy(), vz=zeros.copy(),
        L=np.array([L32], np.float32), vol_off=np.array([0, n], np.int64), **kw)


def uniform_positions(rng: np.random.Generator, n: int, L: float) -> np.ndarray:
    """n positions uniform in [0, L)^3, float64 [n, 3]."""
    return rng.random((n, 3)) * L


def nfw_mu(x):
    """Enclosed-mass shape of the NFW profile, mu(x) = ln(1+x) - x/(1+x)."""
    return np.log1p(x) - x / (1.0 + x)


def nfw_radii(rng: np.random.Generator, n: int, c: float, r_s: float) -> np.ndarray:
    """n radii drawn from an NFW profile truncated at x = c (r = x r_s).

    Inverts mu(x)/mu(c) = u by float64 bisection on [0, c] (60 halvings).
    """
    u = rng.random(n) * nfw_mu(c)
    lo = np.zeros(n)
    hi = np.full(n, float(c))
    for _ in range(60):
        mid = 0.5 * (lo + hi)
        below = nfw_mu(mid) < u
        lo = np.where(below, mid, lo)
        hi = np.where(below, hi, mid)
    return 0.5 * (lo + hi) * r_s


def isotropic_dirs(rng: np.random.Generator, n: int) -> np.ndarray:
    cz = rng.random(n) * 2.0 - 1.0
    phi = rng.random(n) * (2.0 * math.pi)
    sz = np.sqrt(np.maximum(0.0, 1.0 - cz * cz))
    return np.stack([sz * np.cos(phi), sz * np.sin(phi), cz], axis=1)


def halo_counts(rng: np.random.Generator, n_halos: int, budget: int,
                m_lo: float = 1e2, m_hi: float = 1e5) -> np.ndarray:
    """Particle counts of n_halos halos summing to exactly ``budget``.

    Masses are drawn log-uniform on [m_lo, m_hi] particles, then scaled in
    proportion so that they sum to the budget, with largest-remainder rounding
    (the stated halo recipe overshoots the 40 % particle budget otherwise).
    """
    raw = np.exp(rng.uniform(math.log(m_lo), math.log(m_hi), n_halos))
    scaled = raw * (budget / raw.sum())
    counts = np.floor(scaled).astype(np.int64)
    rem = budget - int(counts.sum())
    if rem > 0:
        order = np.argsort(-(scaled - counts), kind="stable")
        counts[order[:rem]] += 1
    return counts


def clustered_positions(rng: np.random.Generator, n: int, L: float, n_halos: int,
                        halo_frac: float = 0.4) -> tuple[np.ndarray, dict]:
    """Uniform background plus NFW halos, float64 [n, 3] (not yet wrapped).

    Draw order: background positions, halo centres, halo masses,
    concentrations, then per halo its radii and directions.
    """
    budget = int(round(halo_frac * n))
    n_bg = n - budget
    bg = uniform_positions(rng, n_bg, L)
    centres = rng.random((n_halos, 3)) * L
    counts = halo_counts(rng, n_halos, budget)
    conc = rng.uniform(5.0, 10.0, n_halos)
    parts = [bg]
    for h in range(n_halos):
        k = int(counts[h])
        if k == 0:
            continue
        r200 = (3.0 * k / (800.0 * math.pi)) ** (1.0 / 3.0)
        r = nfw_radii(rng, k, float(conc[h]), r200 / float(conc[h]))
        d = isotropic_dirs(rng, k)
        parts.append(centres[h] + r[:, None] * d)
    pos = np.concatenate(parts, axis=0)
    return pos, {"halo_counts": counts, "halo_centres": centres, "concentration": conc}


def uniform_box(n: int = 4096, L: float = 16.0, seed: int = 1, **kw) -> Workload:
    """n particles uniform in a periodic box of side L (the small test case)."""
    rng = np.random.default_rng(seed)
    L32 = np.float32(L)
    return _single(f"uniform_{n}_L{L:g}", uniform_positions(rng, n, float(L32)), L32, **kw)


def lattice_zeldovich(side: int = 128, rms: float = 0.5, seed: int = 2, **kw) -> Workload:
    """side^3 particles on a unit lattice (x = i + 0.5) plus Gaussian displacements.

    Each axis gets an independent N(0, rms^2) displacement (a Zel'dovich-style
    perturbed lattice without a power spectrum); box side = side grid units.
    """
    rng = np.random.default_rng(seed)
    g = np.arange(side, dtype=np.float64) + 0.5
    gz, gy, gx = np.meshgrid(g, g, g, indexing="ij")
    pos = np.stack([gx.ravel(), gy.ravel(), gz.ravel()], axis=1)
    if rms > 0:
        pos = pos + rng.normal(0.0, rms, pos.shape)
    return _single(f"lattice_{side}^3_rms{rms:g}", pos, np.float32(side), **kw)


def clustered_box(side: int = 256, n_halos: int = 2000, seed: int = 3, **kw) -> Workload:
    """side^3 particles in a box of side grid units: 60 % uniform, 40 % in NFW halos."""
    rng = np.random.default_rng(seed)
    n = side ** 3
    L32 = np.float32(side)
    pos, info = clustered_positions(rng, n, float(L32), n_halos)
    w = _single(f"clustered_{side}^3_{n_halos}halos", pos, L32, **kw)
    w.extra.update(info)
    return w


def batched_volumes(V: int = 256, n_lo: int = 4096, n_hi: int = 262144, seed: int = 5,
                    **kw) -> Workload:
    """V independent periodic sub-volumes with log-uniform particle counts.

    Volume b holds N_b = round(exp(U(ln n_lo, ln n_hi))) particles in a box of
    side N_b^(1/3) (mean density one per grid cell cubed).  The first half are
    uniform, the second half follow the halo recipe with
    round(max(1, 2000 N_b / 256^3)) halos.
    """
    rng = np.random.default_rng(seed)
    counts = np.rint(np.exp(rng.uniform(math.log(n_lo), math.log(n_hi), V))).astype(np.int64)
    xs, ys, zs, Ls = [], [], [], []
    for b in range(V):
        nb = int(counts[b])
        L32 = np.float32(nb ** (1.0 / 3.0))
        if b < V // 2:
            pos = uniform_positions(rng, nb, float(L32))
        else:
            nh = int(round(max(1.0, 2000.0 * nb / 256 ** 3)))
            pos, _ = clustered_positions(rng, nb, float(L32), nh)
        xs.append(_wrap32(pos[:, 0], L32))
        ys.append(_wrap32(pos[:, 1], L32))
        zs.append(_wrap32(pos[:, 2], L32))
        Ls.append(L32)
    x = np.concatenate(xs)
    n = x.shape[0]
    zeros = np.zeros(n, np.float32)
    vol_off = np.zeros(V + 1, np.int64)
    vol_off[1:] = np.cumsum(counts)
    return Workload(name=f"batched_{V}vols", x=x, y=np.concatenate(ys), z=np.concatenate(zs),
                    m=np.ones(n, np.float32), vx=zeros.copy(), vy=zeros.copy(),
                    vz=zeros.copy(), L=np.array(Ls, np.float32), vol_off=vol_off, **kw)


CONFIG_NAMES = ("uniform4096", "lattice128", "clustered256", "diff64", "batched256")


def make_config(name: str) -> Workload:
    """The five standard workloads of the short-range force benchmark.

    uniform4096  : 4096 uniform particles, L = 16, r_c = 3, eps = 0.01.
    lattice128   : 128^3 perturbed lattice (rms 0.5), L = 128, force + kick (dt 0.01).
    clustered256 : 256^3 particles, 60 % uniform + 40 % in 2000 NFW halos, L = 256.
    diff64       : 64^3 particles, same recipe with 100 halos, L = 64; four
                   kick-drift steps of dt = 0.01 and a loss weighted by seeded
                   N(0, 1) vectors (seed 40).
    batched256   : 256 sub-volumes, 4k-256k particles each.
    """
    if name == "uniform4096":
        return uniform_box(4096, 16.0, seed=1)
    if name == "lattice128":
        return lattice_zeldovich(128, 0.5, seed=2)
    if name == "clustered256":
        return clustered_box(256, 2000, seed=3)
    if name == "diff64":
        w = clustered_box(64, 100, seed=4)
        rng = np.random.default_rng(40)
        w.extra["loss_w"] = rng.normal(0.0, 1.0, (w.N, 3)).astype(np.float32)
        w.extra["steps"] = 4
        return w
    if name == "batched256":
        return batched_volumes(256, seed=5)
    raise KeyError(name)
