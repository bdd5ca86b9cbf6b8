"""The equal-mass path of the force kernels (hacc_binned::mass_varies).

HACC's particles all carry one mass; the binning (and the tree build) flag
that case on the device, and the gather and symmetric force kernels then sum
f d and scale each total by the particle's own mass.  Checked here: the flag
for equal, varied, signed-zero and empty inputs on both list builders; both
kernels against the float64 oracle with a common mass other than one and with
varied masses; and the equal-mass path against the general path (the same
inputs with the flag withheld) to float32 rounding."""

import dataclasses

import numpy as np
import pytest

import oracle
from gpu_util import MAX_TOL, RMS_TOL, err_norms, need_cuda
from synth import default_coeffs, uniform_box
from synth.workloads import Workload, clustered_box

pytestmark = pytest.mark.gpu

EPS, RC = 0.01, 3.0


@pytest.fixture(scope="module")
def hs():
    need_cuda()
    import paper_1211_4864_gb300 as hs
    hs.load()
    return hs


def params(hs):
    return hs.SRParams(EPS, RC, default_coeffs(RC, EPS))


def with_masses(w: Workload, m) -> Workload:
    return dataclasses.replace(w, m=np.asarray(m, np.float32))


def prepare(hs, w: Workload, builder="mesh", equal_mass_path=True, split_T=64):
    import torch
    sr = hs.ShortRange(w.L, w.vol_off, RC, split_T=split_T, builder=builder, equal_mass_path=equal_mass_path)
    pos = torch.tensor(np.stack([w.x, w.y, w.z]), device="cuda")
    m = torch.tensor(w.m, device="cuda")
    sr.prepare(pos, m)
    return sr


def flag(sr) -> int:
    import torch
    torch.cuda.synchronize()
    return int(sr.mass_varies.item())


def forces(hs, sr):
    import torch
    prm = params(hs)
    a_g = sr.force(prm)
    a_s = sr.force_symmetric(prm)
    torch.cuda.synchronize()
    sr.check_status()
    return a_g.cpu().numpy().T.astype(np.float64), a_s.cpu().numpy().T.astype(np.float64)


def oracle_force(w: Workload):
    c = default_coeffs(RC, EPS).astype(np.float64)
    return oracle.sr_force(w.x, w.y, w.z, w.m, float(w.L[0]), EPS, RC, c)


@pytest.mark.parametrize("builder", ["mesh", "rcb"])
def test_mass_flag(hs, builder):
    w = uniform_box(3000, 16.0, seed=11)
    n = w.x.size
    assert flag(prepare(hs, with_masses(w, np.full(n, 0.37)), builder)) == 0
    m = np.full(n, 0.37, np.float32)
    m[-1] = np.nextafter(np.float32(0.37), np.float32(1.0))
    assert flag(prepare(hs, with_masses(w, m), builder)) == 1
    m = np.full(n, 0.0, np.float32)
    m[n // 2] = -0.0  # bitwise different from +0
    assert flag(prepare(hs, with_masses(w, m), builder)) == 1
    rng = np.random.default_rng(2)
    assert flag(prepare(hs, with_masses(w, rng.uniform(0.5, 2.0, n)), builder)) == 1
    # re-binning equal masses clears a flag a previous call set
    sr = prepare(hs, with_masses(w, rng.uniform(0.5, 2.0, n)), builder)
    import torch
    sr.prepare(torch.tensor(np.stack([w.x, w.y, w.z]), device="cuda"), torch.full((n,), 2.0, device="cuda"))
    assert flag(sr) == 0


def test_mass_flag_empty(hs):
    import torch
    sr = hs.ShortRange(np.array([12.0], np.float32), np.array([0, 0], np.int64), RC)
    assert flag(sr) == 1  # nothing binned yet: the general path
    sr.prepare(torch.zeros((3, 0), device="cuda"), torch.zeros(0, device="cuda"))
    assert flag(sr) == 0


@pytest.mark.parametrize("case", ["uniform", "clustered"])
@pytest.mark.parametrize("masses", ["equal", "varied"])
def test_forces_against_oracle(hs, case, masses):
    w = uniform_box(4096, 16.0, seed=1) if case == "uniform" else clustered_box(18, 5, seed=5)
    n = w.x.size
    rng = np.random.default_rng(17)
    w = with_masses(w, np.full(n, 0.37) if masses == "equal" else rng.uniform(0.5, 2.0, n))
    sr = prepare(hs, w)
    assert flag(sr) == (0 if masses == "equal" else 1)
    ref = oracle_force(w)
    a_g, a_s = forces(hs, sr)
    for name, a in (("gather", a_g), ("symmetric", a_s)):
        rms, mx = err_norms(a, ref)
        assert rms < RMS_TOL and mx < MAX_TOL, (name, rms, mx)


@pytest.mark.parametrize("builder", ["mesh", "rcb"])
def test_equal_mass_path_matches_general_path(hs, builder):
    w = clustered_box(20, 6, seed=9)
    w = with_masses(w, np.full(w.x.size, 1.0))
    sr_eq = prepare(hs, w, builder)
    sr_gen = prepare(hs, w, builder, equal_mass_path=False)
    assert flag(sr_eq) == 0 and sr_gen.mass_varies is None
    g_eq, s_eq = forces(hs, sr_eq)
    g_gen, s_gen = forces(hs, sr_gen)
    # unit masses: the two gather paths differ only by the products with 1
    assert np.array_equal(g_eq, g_gen)
    rms, mx = err_norms(s_eq, s_gen)
    assert rms < 1e-6 and mx < MAX_TOL, (rms, mx)
    ref = oracle_force(w)
    for a in (g_eq, s_eq, g_gen, s_gen):
        rms, mx = err_norms(a, ref)
        assert rms < RMS_TOL and mx < MAX_TOL, (rms, mx)


@pytest.mark.parametrize("kernel", ["gather", "symmetric"])
@pytest.mark.parametrize("masses", ["equal", "varied"])
@pytest.mark.parametrize("want_gm", [False, True])
def test_adjoints_against_oracle(hs, kernel, masses, want_gm):
    """Both adjoints on both mass paths, with and without dL/dm, against the
    float64 analytic adjoint."""
    import torch
    w = clustered_box(18, 5, seed=23)
    n = w.x.size
    rng = np.random.default_rng(31)
    w = with_masses(w, np.full(n, 0.37) if masses == "equal" else rng.uniform(0.5, 2.0, n))
    lam = rng.normal(size=(n, 3)).astype(np.float32)
    sr = prepare(hs, w)
    assert flag(sr) == (0 if masses == "equal" else 1)
    prm = params(hs)
    fn = sr.adjoint if kernel == "gather" else sr.adjoint_symmetric
    g, gm = fn(prm, torch.tensor(lam.T.copy(), device="cuda"), want_gm=want_gm)
    torch.cuda.synchronize()
    sr.check_status()
    rg, rgm = oracle.sr_force_adjoint(w.x, w.y, w.z, w.m, float(w.L[0]), EPS, RC,
                                      default_coeffs(RC, EPS).astype(np.float64), lam)
    rms, _ = err_norms(g.cpu().numpy().T, rg)
    assert rms < RMS_TOL, rms
    if want_gm:
        grms = np.linalg.norm(gm.cpu().numpy() - rgm) / np.linalg.norm(rgm)
        assert grms < RMS_TOL, grms


@pytest.mark.parametrize("split_T", [128, 97, 65])
@pytest.mark.parametrize("masses", ["equal", "varied"])
def test_symmetric_adjoint_four_per_lane(hs, split_T, masses):
    """Without dL/dm (the single antisymmetric vector sum per pair) the
    symmetric adjoint runs tasks of 65 to 128 particles with four i per lane
    (the chunk's own four blocks, then the half stencil), on either mass path.
    Against the float64 adjoint and the gather adjoint."""
    import torch
    w = clustered_box(18, 5, seed=29)
    n = w.x.size
    rng = np.random.default_rng(37)
    w = with_masses(w, np.full(n, 0.37) if masses == "equal" else rng.uniform(0.5, 2.0, n))
    lam = rng.normal(size=(n, 3)).astype(np.float32)
    sr = prepare(hs, w, split_T=split_T)
    assert flag(sr) == (0 if masses == "equal" else 1)
    sizes = np.diff(sr.tasks.cpu().numpy()[: int(sr.n_tasks.item()), 1:3], axis=1).ravel()
    assert sizes.max() > 64  # the four-per-lane path runs
    prm = params(hs)
    lt = torch.tensor(lam.T.copy(), device="cuda")
    g_s, _ = sr.adjoint_symmetric(prm, lt, want_gm=False)
    g_g, _ = sr.adjoint(prm, lt, want_gm=False)
    torch.cuda.synchronize()
    sr.check_status()
    rg, _ = oracle.sr_force_adjoint(w.x, w.y, w.z, w.m, float(w.L[0]), EPS, RC,
                                    default_coeffs(RC, EPS).astype(np.float64), lam)
    for name, g in (("symmetric", g_s), ("gather", g_g)):
        rms, _ = err_norms(g.cpu().numpy().T, rg)
        assert rms < RMS_TOL, (name, rms)
