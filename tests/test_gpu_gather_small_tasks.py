"""The gather kernels on tasks of at most 16 particles, which run each i on
two lanes (each lane takes half of every staged piece of j records and the two
compensated partial sums are added at the end).

Split sizes 16, 11 and 1 put every task on that path; 17 and 40 mix it with
the one- and two-i-per-lane paths (a cell's last task is often 16 particles or
fewer).
Checked for the force, the potential and both adjoints, on both mass paths,
against the float64 oracle, and the result of one launch repeated bit for bit."""

import dataclasses

import numpy as np
import pytest

import oracle
from gpu_util import MAX_TOL, RMS_TOL, err_norms, need_cuda
from synth import default_coeffs, uniform_box
from synth.workloads import clustered_box

pytestmark = pytest.mark.gpu

EPS, RC = 0.01, 3.0
SPLITS = [16, 11, 1, 17, 40]


@pytest.fixture(scope="module")
def hs():
    need_cuda()
    import paper_1211_4864_gb300 as hs
    hs.load()
    return hs


@pytest.fixture(scope="module", params=["uniform", "clustered"])
def case(request):
    """Uniform cells of ~24 particles, or clustered cells of up to hundreds,
    with varied masses and one shared cotangent."""
    w = uniform_box(3000, 16.0, seed=41) if request.param == "uniform" else clustered_box(18, 5, seed=43)
    rng = np.random.default_rng(47)
    w = dataclasses.replace(w, m=rng.uniform(0.5, 2.0, w.N).astype(np.float32))
    lam = rng.normal(size=(w.N, 3)).astype(np.float32)
    c = default_coeffs(RC, EPS).astype(np.float64)
    L = float(w.L[0])
    ref = {
        "force": oracle.sr_force(w.x, w.y, w.z, w.m, L, EPS, RC, c),
        "potential": oracle.sr_potential(w.x, w.y, w.z, w.m, L, EPS, RC, c),
        "adjoint": oracle.sr_force_adjoint(w.x, w.y, w.z, w.m, L, EPS, RC, c, lam),
    }
    return w, lam, ref


def run(hs, w, lam, split_T, masses):
    import torch
    m = w.m if masses == "varied" else np.full(w.N, 0.37, np.float32)
    sr = hs.ShortRange(w.L, w.vol_off, RC, split_T=split_T)
    sr.prepare(torch.tensor(np.stack([w.x, w.y, w.z]), device="cuda"), torch.tensor(m, device="cuda"))
    prm = hs.SRParams(EPS, RC, default_coeffs(RC, EPS))
    lt = torch.tensor(lam.T.copy(), device="cuda")
    out = {
        "force": sr.force(prm).cpu().numpy().T.astype(np.float64),
        "force_again": sr.force(prm).cpu().numpy().T.astype(np.float64),
        "potential": sr.potential(prm).cpu().numpy().astype(np.float64),
    }
    g, gm = sr.adjoint(prm, lt, want_gm=True)
    out["adjoint"] = (g.cpu().numpy().T.astype(np.float64), gm.cpu().numpy().astype(np.float64))
    g2, _ = sr.adjoint(prm, lt, want_gm=False)
    out["adjoint_nogm"] = g2.cpu().numpy().T.astype(np.float64)
    torch.cuda.synchronize()
    sr.check_status()
    return out


@pytest.mark.parametrize("split_T", SPLITS)
def test_half_warp_tasks_against_oracle(hs, case, split_T):
    w, lam, ref = case
    got = run(hs, w, lam, split_T, "varied")
    rms, mx = err_norms(got["force"], ref["force"])
    assert rms < RMS_TOL and mx < MAX_TOL, ("force", rms, mx)
    assert np.array_equal(got["force"], got["force_again"])
    phi, rphi = got["potential"], ref["potential"]
    assert np.linalg.norm(phi - rphi) / np.linalg.norm(rphi) < 1e-5
    assert np.max(np.abs(phi - rphi)) < 1e-4 * np.max(np.abs(rphi))
    rg, rgm = ref["adjoint"]
    g, gm = got["adjoint"]
    assert err_norms(g, rg)[0] < RMS_TOL
    assert err_norms(got["adjoint_nogm"], rg)[0] < RMS_TOL
    assert np.linalg.norm(gm - rgm) / np.linalg.norm(rgm) < RMS_TOL


@pytest.mark.parametrize("split_T", [16, 17])
def test_half_warp_tasks_equal_masses(hs, case, split_T):
    """The equal-mass instantiations (mass 0.37 everywhere): the force and
    the adjoint against the oracle on the same masses."""
    w, lam, _ = case
    m = np.full(w.N, 0.37, np.float32)
    c = default_coeffs(RC, EPS).astype(np.float64)
    L = float(w.L[0])
    got = run(hs, w, lam, split_T, "equal")
    rms, mx = err_norms(got["force"], oracle.sr_force(w.x, w.y, w.z, m, L, EPS, RC, c))
    assert rms < RMS_TOL and mx < MAX_TOL, (rms, mx)
    rg, rgm = oracle.sr_force_adjoint(w.x, w.y, w.z, m, L, EPS, RC, c, lam)
    assert err_norms(got["adjoint"][0], rg)[0] < RMS_TOL
    assert err_norms(got["adjoint_nogm"], rg)[0] < RMS_TOL
    assert np.linalg.norm(got["adjoint"][1] - rgm) / np.linalg.norm(rgm) < RMS_TOL
