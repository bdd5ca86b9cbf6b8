"""GPU parity of the Newton-III symmetric pair kernel (hacc_sr_force_symmetric):
the same forces as the gather kernel and the float64 oracle from half the
pair evaluations, on uniform, clustered, fine-mesh, small-box and batched
inputs, every launch shape, and tiny task sizes."""

import numpy as np
import pytest

import oracle
from gpu_util import MAX_TOL, RMS_TOL, err_norms, need_cuda
from synth import default_coeffs, uniform_box
from synth.workloads import Workload, batched_volumes, clustered_box

pytestmark = pytest.mark.gpu

EPS, RC = 0.01, 3.0
SHAPES = [(8, 3, 32, 2), (8, 3, 32, 4), (8, 3, 64, 2), (8, 3, 64, 3), (8, 3, 64, 4), (8, 3, 128, 2),
          (8, 3, 128, 3), (4, 3, 128, 4), (8, 3, 256, 2)]


@pytest.fixture(scope="module")
def hs():
    need_cuda()
    import paper_1211_4864_gb300 as hs
    hs.load()
    return hs


def params(hs):
    return hs.SRParams(EPS, RC, default_coeffs(RC, EPS))


def run_both(hs, w: Workload, cell_min=None, split_T=64, launch=None):
    import torch
    prm = params(hs)
    sr = hs.ShortRange(w.L, w.vol_off, RC, cell_min=cell_min, split_T=split_T)
    pos = torch.tensor(np.stack([w.x, w.y, w.z]), device="cuda")
    m = torch.tensor(w.m, device="cuda")
    sr.prepare(pos, m)
    a_s = sr.force_symmetric(prm, launch=launch)
    a_g = sr.force(prm)
    mom = sr.moments(m, None, a_s).cpu().numpy()
    torch.cuda.synchronize()
    sr.check_status()
    return sr, a_s.cpu().numpy().T.astype(np.float64), a_g.cpu().numpy().T.astype(np.float64), mom


def oracle_force(w: Workload, v=0, targets=None):
    b, e = int(w.vol_off[v]), int(w.vol_off[v + 1])
    c = default_coeffs(RC, EPS).astype(np.float64)
    return oracle.sr_force(w.x[b:e], w.y[b:e], w.z[b:e], w.m[b:e], float(w.L[v]), EPS, RC, c, targets)


@pytest.mark.parametrize("case", ["uniform", "clustered", "fine_mesh", "small_box", "tiny_tasks", "tasks16",
                                  "tasks128", "tasks100"])
def test_symmetric_against_oracle_and_gather(hs, case):
    cell_min, split_T = None, 64
    if case == "uniform":
        w = uniform_box(4096, 16.0, seed=1)
    elif case == "clustered":
        w = clustered_box(20, 4, seed=21)
    elif case == "fine_mesh":  # reach 2: 125 list entries per cell, the forward half spans several groups
        w, cell_min = uniform_box(3000, 14.0, seed=18), 1.5
    elif case == "small_box":  # n = 3 cells per side: every neighbour is a periodic image
        w = uniform_box(1500, 9.0, seed=19)
    elif case == "tiny_tasks":  # chunks of 7 particles: many tasks per cell, every diagonal block ragged
        w, split_T = clustered_box(16, 3, seed=22), 7
    elif case == "tasks16":  # chunks of 16: every task on the half-warp rotation, full halves
        w, split_T = clustered_box(18, 4, seed=24), 16
    elif case == "tasks128":  # four i per lane in the symmetric kernel, 64-particle sub-chunks in the gather
        w, split_T = clustered_box(20, 4, seed=25), 128
    else:  # 100-particle chunks: the fourth i set partly empty
        w, split_T = clustered_box(20, 4, seed=26), 100
    rng = np.random.default_rng(5)
    w.m[:] = rng.uniform(0.5, 1.5, w.N).astype(np.float32)
    sr, a_s, a_g, mom = run_both(hs, w, cell_min=cell_min, split_T=split_T)
    ref = oracle_force(w)
    rms, mx = err_norms(a_s, ref)
    assert rms < RMS_TOL and mx < MAX_TOL, (rms, mx)
    rms, mx = err_norms(a_s, a_g)
    assert rms < 1e-6 and mx < MAX_TOL, (rms, mx)
    # Newton's third law holds by construction: the net force vanishes to float64 rounding of the sums
    assert np.all(np.abs(mom[3:6]) < 1e-6 * mom[7]), mom


@pytest.mark.parametrize("shape", SHAPES)
def test_symmetric_every_launch_shape(hs, shape):
    w = clustered_box(16, 3, seed=23)
    launch = hs.Launch(*shape)
    _, a_s, a_g, _ = run_both(hs, w, launch=launch)
    rms, mx = err_norms(a_s, a_g)
    assert rms < 1e-6 and mx < MAX_TOL, (shape, rms, mx)


def test_symmetric_batched_volumes(hs):
    w = batched_volumes(12, n_lo=800, n_hi=6000, seed=7)
    _, a_s, _, _ = run_both(hs, w)
    for v in range(w.V):
        b, e = int(w.vol_off[v]), int(w.vol_off[v + 1])
        rms, mx = err_norms(a_s[b:e], oracle_force(w, v))
        assert rms < RMS_TOL and mx < MAX_TOL, (v, rms, mx)


def test_symmetric_empty_volume_and_empty_input(hs):
    import torch
    wa, wb = uniform_box(700, 10.0, seed=31), uniform_box(900, 11.0, seed=32)
    cat = lambda f: np.concatenate([getattr(wa, f), getattr(wb, f)])
    w = Workload("gap", cat("x"), cat("y"), cat("z"), cat("m"), cat("vx"), cat("vy"), cat("vz"),
                 np.array([10.0, 9.5, 11.0], np.float32), np.array([0, 700, 700, 1600], np.int64))
    _, a_s, _, _ = run_both(hs, w)
    for v, (b, e) in ((0, (0, 700)), (2, (700, 1600))):
        rms, mx = err_norms(a_s[b:e], oracle_force(w, v))
        assert rms < RMS_TOL and mx < MAX_TOL, (v, rms, mx)
    prm = params(hs)
    sr = hs.ShortRange(np.array([12.0], np.float32), np.array([0, 0], np.int64), RC)
    empty = torch.zeros((3, 0), device="cuda")
    sr.prepare(empty, torch.zeros(0, device="cuda"))
    a = sr.force_symmetric(prm)
    torch.cuda.synchronize()
    sr.check_status()
    assert a.shape == (3, 0)


@pytest.mark.parametrize("case,leaf_max", [("uniform", 32), ("clustered", 64), ("clustered", 7)])
def test_symmetric_on_tree_lists(hs, case, leaf_max):
    """The symmetric force and adjoint on RCB leaf lists (own entry found by
    bisection, forward half after it) against the oracle and the gather
    kernels on the same lists."""
    import torch
    w = uniform_box(3000, 12.0, seed=3) if case == "uniform" else clustered_box(20, 4, seed=24)
    rng = np.random.default_rng(12)
    w.m[:] = rng.uniform(0.5, 1.5, w.N).astype(np.float32)
    prm = params(hs)
    sr = hs.ShortRange(w.L, w.vol_off, RC, split_T=64, builder="rcb", leaf_max=leaf_max)
    m = torch.tensor(w.m, device="cuda")
    sr.prepare(torch.tensor(np.stack([w.x, w.y, w.z]), device="cuda"), m)
    a_s = sr.force_symmetric(prm)
    a_g = sr.force(prm)
    lam = rng.normal(size=(w.N, 3)).astype(np.float32)
    lt = torch.tensor(lam.T.copy(), device="cuda")
    g_s, gm_s = sr.adjoint_symmetric(prm, lt)
    mom = sr.moments(m, None, a_s).cpu().numpy()
    torch.cuda.synchronize()
    sr.check_status()
    S = a_s.cpu().numpy().T.astype(np.float64)
    rms, mx = err_norms(S, oracle_force(w))
    assert rms < RMS_TOL and mx < MAX_TOL, (rms, mx)
    rms, mx = err_norms(S, a_g.cpu().numpy().T.astype(np.float64))
    assert rms < 1e-6 and mx < MAX_TOL, (rms, mx)
    assert np.all(np.abs(mom[3:6]) < 1e-6 * mom[7]), mom
    c = default_coeffs(RC, EPS).astype(np.float64)
    rg, rgm = oracle.sr_force_adjoint(w.x, w.y, w.z, w.m, float(w.L[0]), EPS, RC, c, lam)
    rms, _ = err_norms(g_s.cpu().numpy().T, rg)
    assert rms < RMS_TOL, rms
    assert np.linalg.norm(gm_s.cpu().numpy() - rgm) / np.linalg.norm(rgm) < RMS_TOL


@pytest.mark.parametrize("case,want_gm", [("uniform", True), ("clustered", True), ("clustered", False),
                                          ("fine_mesh", True), ("tiny_tasks", True), ("tasks128", True)])
def test_symmetric_adjoint_against_oracle_and_gather(hs, case, want_gm):
    import torch
    cell_min, split_T = None, 64
    if case == "uniform":
        w = uniform_box(4096, 16.0, seed=1)
    elif case == "clustered":
        w = clustered_box(20, 4, seed=21)
    elif case == "fine_mesh":
        w, cell_min = uniform_box(3000, 14.0, seed=18), 1.5
    elif case == "tasks128":  # both adjoints walk 128-particle tasks in 64-particle sub-chunks
        w, split_T = clustered_box(20, 4, seed=25), 128
    else:
        w, split_T = clustered_box(16, 3, seed=22), 7
    rng = np.random.default_rng(9)
    w.m[:] = rng.uniform(0.5, 1.5, w.N).astype(np.float32)
    lam = rng.normal(size=(w.N, 3)).astype(np.float32)
    prm = params(hs)
    sr = hs.ShortRange(w.L, w.vol_off, RC, cell_min=cell_min, split_T=split_T)
    sr.prepare(torch.tensor(np.stack([w.x, w.y, w.z]), device="cuda"), torch.tensor(w.m, device="cuda"))
    lt = torch.tensor(lam.T.copy(), device="cuda")
    gs, gms = sr.adjoint_symmetric(prm, lt, want_gm=want_gm)
    gg, gmg = sr.adjoint(prm, lt, want_gm=want_gm)
    torch.cuda.synchronize()
    sr.check_status()
    S, G = gs.cpu().numpy().T.astype(np.float64), gg.cpu().numpy().T.astype(np.float64)
    c = default_coeffs(RC, EPS).astype(np.float64)
    ref, rgm = oracle.sr_force_adjoint(w.x, w.y, w.z, w.m, float(w.L[0]), EPS, RC, c, lam)
    # gradients are held to the rms tolerance, as the gather adjoint's parity test holds them
    rms, _ = err_norms(S, ref)
    assert rms < RMS_TOL, rms
    # the gather adjoint itself is ~2e-6 rms from the oracle (the final m U - lam V + X cancels), so the
    # two float32 results are compared at the oracle tolerance
    rms, _ = err_norms(S, G)
    assert rms < RMS_TOL, rms
    # a translation-invariant loss: the position gradient sums to zero
    assert np.linalg.norm(S.sum(0)) < 1e-6 * np.abs(S).sum()
    if want_gm:
        got = gms.cpu().numpy().astype(np.float64)
        assert np.linalg.norm(got - rgm) / np.linalg.norm(rgm) < RMS_TOL
        assert np.linalg.norm(got - gmg.cpu().numpy()) / np.linalg.norm(rgm) < RMS_TOL
    else:
        assert gms is None


@pytest.mark.parametrize("shape", [(8, 2, 32, 2), (8, 2, 64, 4), (8, 2, 128, 2), (4, 2, 128, 3), (8, 1, 256, 2)])
def test_symmetric_adjoint_launch_shapes(hs, shape):
    import torch
    w = clustered_box(16, 3, seed=23)
    rng = np.random.default_rng(10)
    lt = torch.tensor(rng.normal(size=(3, w.N)).astype(np.float32), device="cuda")
    prm = params(hs)
    sr = hs.ShortRange(w.L, w.vol_off, RC, split_T=64)
    sr.prepare(torch.tensor(np.stack([w.x, w.y, w.z]), device="cuda"), torch.tensor(w.m, device="cuda"))
    gs, _ = sr.adjoint_symmetric(prm, lt, launch=hs.Launch(*shape))
    gg, _ = sr.adjoint(prm, lt)
    torch.cuda.synchronize()
    sr.check_status()
    rms, _ = err_norms(gs.cpu().numpy().T, gg.cpu().numpy().T.astype(np.float64))
    assert rms < RMS_TOL, (shape, rms)
