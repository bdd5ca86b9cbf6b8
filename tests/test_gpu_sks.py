"""Short-range sub-cycles of the split-operator step (Eq. 6): potential,
energies, and S(h/2) K(h) S(h/2) trajectories against the float64 oracle,
eager and replayed from a CUDA graph."""

import numpy as np
import pytest

import oracle
from gpu_util import need_cuda
from oracle import sks
from synth import default_coeffs, uniform_box
from synth.workloads import clustered_box

pytestmark = pytest.mark.gpu

EPS, RC = 0.01, 3.0


@pytest.fixture(scope="module")
def hs():
    need_cuda()
    import paper_1211_4864_gb300 as hs
    hs.load()
    return hs


@pytest.mark.parametrize("maker", ["uniform", "clustered"])
def test_potential_against_oracle(hs, maker):
    import torch
    w = uniform_box(4096, 16.0, seed=1) if maker == "uniform" else clustered_box(20, 4, seed=21)
    rng = np.random.default_rng(3)
    w.m[:] = rng.uniform(0.5, 1.5, w.N).astype(np.float32)
    prm = hs.SRParams(EPS, RC, default_coeffs(RC, EPS))
    sr = hs.ShortRange(w.L, w.vol_off, RC, split_T=64)
    pos = torch.tensor(np.stack([w.x, w.y, w.z]), device="cuda")
    m = torch.tensor(w.m, device="cuda")
    sr.prepare(pos, m)
    phi = sr.potential(prm)
    mom = sr.moments(m, None, None, phi).cpu().numpy()
    torch.cuda.synchronize()
    sr.check_status()
    ref = oracle.sr_potential(w.x, w.y, w.z, w.m, float(w.L[0]), EPS, RC, prm.c.astype(np.float64))
    got = phi.cpu().numpy().astype(np.float64)
    assert np.linalg.norm(got - ref) / np.linalg.norm(ref) < 1e-5
    assert np.max(np.abs(got - ref)) < 1e-4 * np.max(np.abs(ref))
    e_ref = 0.5 * np.sum(w.m.astype(np.float64) * ref)
    assert mom[8] == pytest.approx(e_ref, rel=1e-5)


def test_sks_subcycles_against_oracle_eager_and_graph(hs):
    import torch
    w = uniform_box(4096, 16.0, seed=1)
    rng = np.random.default_rng(4)
    v0 = (rng.normal(size=(w.N, 3)) * 0.3).astype(np.float32)
    prm = hs.SRParams(EPS, RC, default_coeffs(RC, EPS))
    h, n_c = 0.002, 8
    x0 = np.stack([w.x, w.y, w.z], 1)

    sr = hs.ShortRange(w.L, w.vol_off, RC, split_T=64)
    m = torch.tensor(w.m, device="cuda")
    pos = torch.tensor(x0.T.copy(), device="cuda")
    v = torch.tensor(v0.T.copy(), device="cuda")
    # the acceleration buffer's old contents must not matter (the stream maps never read it)
    a = torch.full_like(v, float("nan"))
    sr.sks_subcycles(pos, v, m, prm, h, n_c, a)
    sr.prepare(pos, m)
    phi = sr.potential(prm)
    mom = sr.moments(m, v, None, phi).cpu().numpy()
    torch.cuda.synchronize()
    sr.check_status()
    P, V = pos.cpu().numpy().T.astype(np.float64), v.cpu().numpy().T.astype(np.float64)

    xr, vr, hist = sks.subcycles(x0, v0, w.m, float(w.L[0]), EPS, RC, prm.c.astype(np.float64), h, n_c)
    dx = P - xr
    dx -= 16.0 * np.round(dx / 16.0)
    assert np.max(np.abs(dx)) < 2e-5
    assert np.max(np.abs(V - vr)) < 1e-4 * np.max(np.abs(vr))
    ke, pe = hist[-1]
    assert mom[6] == pytest.approx(ke, rel=1e-5)
    assert mom[8] == pytest.approx(pe, rel=1e-5)

    # the same sub-cycles captured once and replayed: identical to eager
    pos2 = torch.tensor(x0.T.copy(), device="cuda")
    v2 = torch.tensor(v0.T.copy(), device="cuda")
    a2 = torch.empty_like(v2)
    sr.sks_subcycles(pos2, v2, m, prm, h, 1, a2)  # warm-up outside capture
    pos2.copy_(torch.tensor(x0.T.copy(), device="cuda"))
    v2.copy_(torch.tensor(v0.T.copy(), device="cuda"))
    s = torch.cuda.Stream()
    s.wait_stream(torch.cuda.current_stream())
    g = torch.cuda.CUDAGraph()
    with torch.cuda.stream(s):
        pos_in, v_in = pos2.clone(), v2.clone()
        with torch.cuda.graph(g, stream=s):
            sr.sks_subcycles(pos2, v2, m, prm, h, n_c, a2)
    torch.cuda.current_stream().wait_stream(s)
    pos2.copy_(pos_in)
    v2.copy_(v_in)
    g.replay()
    torch.cuda.synchronize()
    sr.check_status()
    assert torch.equal(pos2, pos) and torch.equal(v2, v)


def test_drifted_offsets_give_the_forces_of_a_rebinning(hs):
    """Streaming the binned records (offsets += dt v) and reusing lists built
    for r_c + skin gives the forces of a fresh binning of the streamed
    positions (to float32 rounding: the offsets are formed differently)."""
    import torch
    w = uniform_box(4096, 16.0, seed=2)
    rng = np.random.default_rng(5)
    v = torch.tensor((rng.normal(size=(3, w.N)) * 0.15).astype(np.float32), device="cuda")
    prm = hs.SRParams(EPS, RC, default_coeffs(RC, EPS))
    m = torch.tensor(w.m, device="cuda")
    pos = torch.tensor(np.stack([w.x, w.y, w.z]), device="cuda")
    sr = hs.ShortRange(w.L, w.vol_off, RC, split_T=64, skin=0.4)
    sr.prepare(pos, m)
    dt = 0.2  # displacements of 0.03 rms, at most ~0.14 < skin / 2
    sr.drift_offsets(v, dt)
    a_drift = sr.force(prm)
    a_sym = sr.force_symmetric(prm)
    torch.cuda.synchronize()
    sr.check_status()
    sr.stream(v, pos, dt)
    fresh = hs.ShortRange(w.L, w.vol_off, RC, split_T=64)
    fresh.prepare(pos, m)
    a_fresh = fresh.force(prm)
    torch.cuda.synchronize()
    fresh.check_status()
    A = a_fresh.cpu().numpy().T.astype(np.float64)
    for a in (a_drift, a_sym):
        got = a.cpu().numpy().T.astype(np.float64)
        assert np.linalg.norm(got - A) / np.linalg.norm(A) < 1e-5
    P = pos.cpu().numpy()
    ref = oracle.sr_force(P[0], P[1], P[2], w.m, 16.0, EPS, RC, prm.c.astype(np.float64))
    assert np.linalg.norm(a_drift.cpu().numpy().T - ref) / np.linalg.norm(ref) < 1e-5


def test_leaving_the_skin_is_flagged(hs):
    import torch
    w = uniform_box(2000, 16.0, seed=3)
    sr = hs.ShortRange(w.L, w.vol_off, RC, split_T=64, skin=0.2)
    sr.prepare(torch.tensor(np.stack([w.x, w.y, w.z]), device="cuda"), torch.tensor(w.m, device="cuda"))
    v = torch.zeros((3, w.N), device="cuda")
    sr.drift_offsets(v, 1.0)  # no motion: inside the skin
    assert hs.hacc_get_status(sr.status) == 0
    v[0, 17] = 1.0
    sr.drift_offsets(v, 3.5)  # one particle moves by more than a cell
    assert hs.hacc_get_status(sr.status) & 8
    with pytest.raises(hs.HaccError):
        sr.check_status()


def test_sks_with_rebinning_every_fifth_subcycle(hs):
    """Sub-cycles that re-bin only every fifth time (lists for r_c + skin,
    binned offsets streamed in between) follow the float64 oracle as closely
    as the re-binning sub-cycles, eager and replayed from a CUDA graph."""
    import torch
    w = uniform_box(4096, 16.0, seed=1)
    rng = np.random.default_rng(4)
    v0 = (rng.normal(size=(w.N, 3)) * 0.3).astype(np.float32)
    prm = hs.SRParams(EPS, RC, default_coeffs(RC, EPS))
    h, n_c = 0.002, 12
    x0 = np.stack([w.x, w.y, w.z], 1)
    sr = hs.ShortRange(w.L, w.vol_off, RC, split_T=64, skin=0.1)
    m = torch.tensor(w.m, device="cuda")
    pos = torch.tensor(x0.T.copy(), device="cuda")
    v = torch.tensor(v0.T.copy(), device="cuda")
    a = torch.empty_like(v)
    sr.sks_subcycles(pos, v, m, prm, h, n_c, a, rebin_every=5)
    torch.cuda.synchronize()
    sr.check_status()
    P, V = pos.cpu().numpy().T.astype(np.float64), v.cpu().numpy().T.astype(np.float64)
    xr, vr, _ = sks.subcycles(x0, v0, w.m, float(w.L[0]), EPS, RC, prm.c.astype(np.float64), h, n_c)
    dx = P - xr
    dx -= 16.0 * np.round(dx / 16.0)
    assert np.max(np.abs(dx)) < 2e-5
    assert np.max(np.abs(V - vr)) < 1e-4 * np.max(np.abs(vr))

    pos2 = torch.tensor(x0.T.copy(), device="cuda")
    v2 = torch.tensor(v0.T.copy(), device="cuda")
    a2 = torch.empty_like(v2)
    s = torch.cuda.Stream()
    s.wait_stream(torch.cuda.current_stream())
    g = torch.cuda.CUDAGraph()
    with torch.cuda.stream(s):
        pos_in, v_in = pos2.clone(), v2.clone()
        with torch.cuda.graph(g, stream=s):
            sr.sks_subcycles(pos2, v2, m, prm, h, n_c, a2, rebin_every=5)
    torch.cuda.current_stream().wait_stream(s)
    pos2.copy_(pos_in)
    v2.copy_(v_in)
    g.replay()
    torch.cuda.synchronize()
    sr.check_status()
    assert torch.equal(pos2, pos) and torch.equal(v2, v)
